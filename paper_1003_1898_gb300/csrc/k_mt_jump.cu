// k_mt_jump.cu -- MT19937 jump-ahead over GF(2) (Section 3.7; Appendix A,
// "Mersenne twister"), host side.
//
// A handle's table of 624 words is a window of the word sequence
// w_{t+624} = w_{t+397} ^ (w_t^upper | w_{t+1}^lower) A, the next outputs
// being tempered words of it; k outputs later the table is the window k
// words further on, with the read index unchanged.  Moving the window by one
// word is a linear map T over GF(2) whose characteristic polynomial phi has
// degree 19937.  On the state, T^k acts as g(T) for g = t^k mod phi; T drops
// the low 31 bits of the window's oldest word (not part of the state), so
// the jump applies g = t^(k-1) mod phi and then one more step, which makes
// every word of the new table exact (the device kernel, k_mt_poly_apply,
// does both at once).
//
//  * phi is found once per process by the Berlekamp-Massey algorithm on
//    2 x 19937 output bits of a host MT19937, with bit-packed polynomials.
//  * t^(k-1) mod phi: left-to-right square-and-multiply, squaring by
//    spreading bits, reduction 64 coefficients at a time using phi's 135
//    terms (its second-highest exponent is 623 below the top, so a 64-bit
//    chunk of high coefficients never lands in itself).
//  * The single-sequence fill from init_genrand(x0): chunk starts by
//    log2(C) doubling passes of the polynomial for (L 2^i), then the
//    ordinary MT19937 fill kernel with one chunk per warp.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "batch.cuh"
#include "scratch.cuh"

namespace prng {

namespace {

constexpr int kD = 19937;             // degree of phi
constexpr int kW = 2 * kD / 64 + 2;   // words of a product before reduction

// Host MT19937: init_genrand and one output.
struct HostMt {
  uint32_t mt[624];
  int mti = 624;
  void init(uint32_t s) {
    mt[0] = s;
    for (int i = 1; i < 624; i++) mt[i] = 1812433253u * (mt[i - 1] ^ (mt[i - 1] >> 30)) + (uint32_t)i;
    mti = 624;
  }
  uint32_t next() {
    if (mti >= 624) {
      for (int k = 0; k < 624; k++) {
        const uint32_t y = (mt[k] & 0x80000000u) | (mt[(k + 1) % 624] & 0x7FFFFFFFu);
        mt[k] = mt[(k + 397) % 624] ^ (y >> 1) ^ ((y & 1u) ? 0x9908B0DFu : 0u);
      }
      mti = 0;
    }
    uint32_t t = mt[mti++];
    t ^= t >> 11;
    t ^= (t << 7) & 0x9D2C5680u;
    t ^= (t << 15) & 0xEFC60000u;
    t ^= t >> 18;
    return t;
  }
};

inline bool bit(const uint64_t* a, int64_t i) { return (a[i >> 6] >> (i & 63)) & 1u; }

// 64 bits of a starting at bit position pos (words past the end read as 0
// are the caller's padding).
inline uint64_t bits64(const uint64_t* a, int64_t pos) {
  const int64_t q = pos >> 6;
  const int sh = (int)(pos & 63);
  return sh ? (a[q] >> sh) | (a[q + 1] << (64 - sh)) : a[q];
}

// a ^= c placed at bit offset q; bits of c that would fall below 0 must be 0.
inline void xor_at(uint64_t* a, uint64_t c, int64_t q) {
  if (q < 0) {
    c >>= -q;
    q = 0;
  }
  const int64_t w = q >> 6;
  const int sh = (int)(q & 63);
  a[w] ^= c << sh;
  if (sh) a[w + 1] ^= c >> (64 - sh);
}

// The exponents of phi's nonzero terms, ascending (the last is kD).
const std::vector<int>& phi_terms() {
  static std::vector<int> terms;
  static std::once_flag once;
  std::call_once(once, [] {
    const int N = 2 * kD;
    const int NW = N / 64 + 4;
    std::vector<uint64_t> R(2 * NW + 4, 0), C(NW, 0), B(NW, 0), T(NW, 0);
    HostMt mt;
    mt.init(5489u);
    for (int n = 0; n < N; n++)           // R holds the sequence reversed
      if (mt.next() & 1u) R[(N - 1 - n) >> 6] |= 1ull << ((N - 1 - n) & 63);
    // Berlekamp-Massey: d_n = sum_{i=0..L} C_i s_{n-i} = parity(C & (R >> (N-1-n))).
    int L = 0, m = 1;
    C[0] = B[0] = 1;
    for (int n = 0; n < N; n++) {
      const int64_t off = N - 1 - n;
      uint64_t d = 0;
      for (int w = 0; w <= L / 64; w++) d ^= C[w] & bits64(R.data(), off + 64 * w);
      if (!(__builtin_popcountll(d) & 1)) {
        m++;
        continue;
      }
      const bool grow = 2 * L <= n;
      if (grow) T = C;
      for (int w = 0; w * 64 + m < N + 64 && w < NW; w++)
        if (B[w]) xor_at(C.data(), B[w], 64 * (int64_t)w + m);
      if (grow) {
        L = n + 1 - L;
        B = T;
        m = 1;
      } else {
        m++;
      }
    }
    for (int e = 0; e <= L; e++)          // phi(t) = t^L C(1/t)
      if (bit(C.data(), L - e)) terms.push_back(e);
  });
  return terms;
}

// r mod phi, for r with coefficients up to bit `top` (kW words).
void reduce(uint64_t* r, int top) {
  const std::vector<int>& terms = phi_terms();
  const int lo_word = kD >> 6;
  for (int w = top >> 6; w >= lo_word; w--) {
    uint64_t c = r[w];
    if (w == lo_word) c &= ~((1ull << (kD & 63)) - 1);   // coefficients below kD stay
    if (!c) continue;
    r[w] ^= c;
    for (size_t j = 0; j + 1 < terms.size(); j++) xor_at(r, c, 64 * (int64_t)w - kD + terms[j]);
  }
}

// r = g^2 mod phi, times t (mod phi) when times_t; g and r have kW words.
void square_mod(const uint64_t* g, uint64_t* r, bool times_t) {
  std::fill(r, r + kW, 0ull);
  for (int w = 0; w <= (kD - 1) / 64; w++) {    // square: coefficient i -> 2 i
    for (int half = 0; half < 2; half++) {
      uint64_t x = (g[w] >> (32 * half)) & 0xFFFFFFFFull;
      x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
      x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
      x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
      x = (x | (x << 2)) & 0x3333333333333333ull;
      x = (x | (x << 1)) & 0x5555555555555555ull;
      r[2 * w + half] = x;
    }
  }
  reduce(r, 2 * kD - 2);
  if (times_t) {
    for (int w = kW - 1; w > 0; w--) r[w] = (r[w] << 1) | (r[w - 1] >> 63);
    r[0] <<= 1;
    reduce(r, kD);
  }
}

// t^e mod phi as a packed polynomial of kW words.
void pow_t(uint64_t e, uint64_t* g) {
  std::fill(g, g + kW, 0ull);
  g[0] = 1;
  int b = 63;
  while (b >= 0 && !((e >> b) & 1)) b--;
  std::vector<uint64_t> r(kW);
  for (; b >= 0; b--) {
    square_mod(g, r.data(), (e >> b) & 1);
    std::copy(r.begin(), r.end(), g);
  }
}

MtPoly device_form(const uint64_t* g) {
  MtPoly p;
  for (int i = 0; i < 624; i++) p.w[i] = (uint32_t)(g[i / 2] >> (32 * (i & 1)));
  return p;
}

// The device form of t^(k-1) mod phi, k >= 1, from a bounded cache (a jump
// fill needs one polynomial per doubling pass).  A miss whose k is even and
// whose k / 2 is cached takes one squaring: t^(k-1) = t (t^(k/2-1))^2.
MtPoly jump_poly(uint64_t k) {
  static std::mutex lock;
  static std::unordered_map<uint64_t, MtPoly> cache;
  std::lock_guard<std::mutex> guard(lock);
  auto it = cache.find(k);
  if (it != cache.end()) return it->second;
  std::vector<uint64_t> g(kW, 0ull);
  auto half = (k % 2 == 0) ? cache.find(k / 2) : cache.end();
  if (half != cache.end()) {
    std::vector<uint64_t> h(kW, 0ull);
    for (int i = 0; i < 624; i++) h[i / 2] |= (uint64_t)half->second.w[i] << (32 * (i & 1));
    square_mod(h.data(), g.data(), true);
  } else {
    pow_t(k - 1, g.data());
  }
  if (cache.size() >= 256) cache.clear();
  return cache.emplace(k, device_form(g.data())).first->second;
}

}  // namespace

cudaError_t launch_skip_mt(uint32_t* state, uint64_t n, uint64_t k, cudaStream_t s) {
  if (n == 0 || k == 0) return cudaSuccess;
  return launch_mt_poly_apply(jump_poly(k), state, 0, n, 0, s);
}

cudaError_t launch_jump_mt(uint64_t x0, uint64_t first, uint64_t n, uint32_t n_chunks,
                           void* d_out, int mode, cudaStream_t s) {
  // Every chunk costs one application of a jump polynomial, the bulk of the
  // call.  A warp per chunk (the fill's full-warp tile) keeps the GPU as busy
  // as two chunks per warp do, so more chunks than that many warps (27 per
  // SM, one wave) are merged into longer ones: any contiguous cut of the one
  // sequence gives the same output.
  const uint32_t wave = 27u * (uint32_t)sm_count();
  Tile tile = default_tile(MT19937, 0);
  if (n_chunks > wave) {
    n_chunks = wave;
    tile = Tile{64, 624, 1};
  }
  const uint64_t L = (n + n_chunks - 1) / n_chunks;   // draws per chunk
  const uint64_t C = (n + L - 1) / L;                 // chunks, none empty
  HostMt mt;
  mt.init((uint32_t)x0);
  uint32_t* S = nullptr;
  cudaError_t e = scratch_alloc(reinterpret_cast<void**>(&S), C * 624 * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(S, mt.mt, sizeof(mt.mt), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && first > 0)   // the start table moved `first` words on, in place
    e = launch_mt_poly_apply(jump_poly(first), S, 0, 1, 0, s);
  // Pass i: chunks [2^i, 2^(i+1)) from chunks [0, 2^i), L 2^i outputs on.
  int i = 0;
  for (uint64_t half = 1; e == cudaSuccess && half < C; half <<= 1, i++)
    e = launch_mt_poly_apply(jump_poly(L << i), S, half, std::min(2 * half, C), half, s);
  if (e == cudaSuccess) {
    FillDesc d{};
    d.state = S;
    d.n_rows = C;
    d.n_per = L;
    d.out = d_out;
    d.pitch = L;
    d.limit = n;
    d.pos = 624;          // fresh tables: the next output twists
    d.mode = mode;
    e = launch_fill_mt(d, tile, s);
  }
  const cudaError_t ef = scratch_free(S, s);
  return e != cudaSuccess ? e : ef;
}

}  // namespace prng
