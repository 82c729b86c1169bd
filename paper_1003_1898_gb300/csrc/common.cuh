// common.cuh -- internal definitions shared by the libprng kernels.
//
// Device-state layouts (all uint32 words):
//   GGL      SoA [1][n]   x
//   XOR128   SoA [4][n]   x, y, z, w
//   RANECU   SoA [2][n]   s1, s2
//   RANMAR   SoA [98][n]  V[0..96], C  -- V is the lag table in canonical order
//                                         V[k] = U[i97 - k] (indices mod 97), so
//                                         V[0] is the next entry overwritten and
//                                         V[64] = U[j97] (Section 3.5; Appendix A,
//                                         "RANMAR")
//   RANLUX   SoA [25][n]  V[0..23], carry -- V[j] = x_{n-24+j}, oldest first
//                                         (Appendix A, "AWC and SWB"); the
//                                         position inside the luxury cycle is
//                                         uniform over streams and lives in the
//                                         handle
//   MT19937  AoS [n][624] mt[0..623]     -- the read index mti is uniform over
//                                         streams and lives in the handle
// SoA keeps every per-thread state load/store coalesced; MT19937 is handled
// one warp per stream, so its table is contiguous per stream instead.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace prng {

enum Gen : int { GGL = 0, XOR128 = 1, RANECU = 2, RANMAR = 3, RANLUX = 4, MT19937 = 5 };

constexpr int kWords[6] = {1, 4, 2, 98, 25, 624};

// Output of a fill.  OUT_F64 turns each pair of consecutive draws into one
// double (reading R11): the kernels run the u32 pipeline over 2 n draws
// per stream and convert each aligned pair (u32 slots 2k, 2k+1) into the
// double that occupies the same 8 bytes.
// OUT_ISING consumes each draw in place (see IsingSink) instead of storing it.
enum OutMode : int { OUT_U32 = 0, OUT_F32 = 1, OUT_F64 = 2, OUT_ISING = 3 };

// Calls fn(std::integral_constant<int, mode>) for a run-time mode.
template <class Fn>
inline auto with_mode(int mode, Fn&& fn) {
  switch (mode) {
    case OUT_F64: return fn(std::integral_constant<int, OUT_F64>{});
    case OUT_F32: return fn(std::integral_constant<int, OUT_F32>{});
    case OUT_ISING: return fn(std::integral_constant<int, OUT_ISING>{});
    default: return fn(std::integral_constant<int, OUT_U32>{});
  }
}

// The consumer of a fused Metropolis half-sweep (OUT_ISING): the draw for
// the site of colour rank k of an L x L checkerboard lattice updates that
// site at once instead of being stored.
struct IsingSink {
  int8_t* spins;       // L x L, row-major, +1/-1
  uint32_t L, half;    // side, L / 2
  uint32_t lg_half;    // log2(half) when half is a power of two, else 32
  uint32_t colour;     // sites with (x + y) % 2 == colour
  uint32_t shift;      // 24-bit acceptance value = draw >> shift
  uint32_t t4, t8;     // integer thresholds for dE = 4 and dE = 8
  uint32_t vec4;       // L % 8 == 0 and spins 8-byte aligned: 4 aligned ranks as one 8-byte chunk
};

// One fill (or skip, or jump fill) as the kernels see it.
struct FillDesc {
  uint32_t* state;     // device state (layout above); unused for jump fills
  uint64_t n_rows;     // streams (or jump chunks)
  uint64_t n_per;      // draws per row in this call
  void* out;           // u32 or f32 output, NULL for a skip
  uint64_t pitch;      // elements between consecutive rows of `out`
  uint64_t limit;      // only elements with linear index < limit are written
  uint64_t x0;         // jump fills: start value (RANECU: s1 | s2 << 32)
  uint32_t pos;        // RANLUX: draws delivered from the current block; MT: mti
  int32_t p;           // RANLUX luxury p
  int32_t mode;        // OutMode: u32 words, floats, or doubles from pairs
  int32_t jump;        // 1: rows are chunks of one jump-ahead sequence
  IsingSink ising;     // OUT_ISING: where element k (= colour rank k) goes
};

// Launch configuration of a fill kernel (chosen by the tuner or defaults).
struct Tile {
  int threads;   // threads per CTA (streams per CTA for thread-per-stream kernels)
  int cols;      // staged columns per tile
  int stages;    // staging buffers (1 or 2)
};

cudaError_t launch_fill_simple(int gen, const FillDesc& d, Tile t, cudaStream_t s);
cudaError_t launch_fill_mlcg(int gen, const FillDesc& d, Tile t, cudaStream_t s);
cudaError_t launch_fill_ranmar(const FillDesc& d, Tile t, cudaStream_t s);
cudaError_t launch_fill_ranlux(const FillDesc& d, Tile t, cudaStream_t s);
cudaError_t launch_fill_mt(const FillDesc& d, Tile t, cudaStream_t s);
cudaError_t launch_seed(int gen, int p, uint64_t seed, uint64_t n, uint32_t* state,
                        cudaStream_t s);
cudaError_t launch_skip_mlcg(int gen, uint32_t* state, uint64_t n, uint64_t k,
                             cudaStream_t s);

Tile default_tile(int gen, int p);

// SplitMix64 (Steele, Lea, Flood 2014): gamma increment, then mix64.
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// MT19937 jump-ahead over GF(2): a polynomial g of degree < 19937 over GF(2)
// (bit i of word i / 32 is the coefficient of t^i) applied to tables of
// 624 words; prng_skip of k outputs on a handle's tables ([n][624]); the
// single-sequence chunked fill from init_genrand(x0).
struct MtPoly {
  uint32_t w[624];
};
cudaError_t launch_mt_poly_apply(const MtPoly& g, uint32_t* state, uint64_t r0, uint64_t r1,
                                 uint64_t src_off, cudaStream_t s);
cudaError_t launch_skip_mt(uint32_t* state, uint64_t n, uint64_t k, cudaStream_t s);
cudaError_t launch_jump_mt(uint64_t x0, uint64_t first, uint64_t n, uint32_t n_chunks,
                           void* d_out, int mode, cudaStream_t s);

// XOR128 jump-ahead over GF(2): prng_skip of k steps on a handle's state
// (struct-of-arrays [4][n]), and the single-sequence chunked fill.
cudaError_t launch_skip_xor128(uint32_t* state, uint64_t n, uint64_t k, cudaStream_t s);
cudaError_t launch_jump_xor128(uint64_t x0, uint64_t first, uint64_t n, uint32_t n_chunks,
                               void* d_out, int f32, cudaStream_t s);

// ------------------------------------------------------------------ device

__device__ __forceinline__ uint32_t umin32(uint32_t a, uint32_t b) { return a < b ? a : b; }

// x <- A x mod (2^31 - C) for a multiplier A < 2^16 and a small C.  With
// p = A x = hi 2^31 + lo31, 2^31 = C (mod m) gives A x = lo31 + C hi, which
// is below 2^31 + 2^24, so one conditional subtraction (unsigned min) ends
// the reduction.  hi = umulhi(x, 2A), and lo31 + C hi = (A x mod 2^32) -
// hi m (mod 2^32), so the fold is three multiply-adds and only the final
// subtraction and min use the integer ALU.  Same integer as the paper's
// Schrage evaluation (Appendix A, eq. RANECU1), other route.
template <uint32_t A, uint32_t C>
__device__ __forceinline__ uint32_t mlcg_step(uint32_t x) {
  constexpr uint32_t M = 0x80000000u - C;
  const uint32_t lo = x * A;
  const uint32_t hi = __umulhi(x, 2u * A);
  const uint32_t r = lo - hi * M;
  return umin32(r, r - M);
}

// x y mod (2^31 - C) for arbitrary x, y < 2^31 (two folds).
template <uint32_t C>
__device__ __forceinline__ uint32_t mulmod_pm(uint32_t x, uint32_t y) {
  constexpr uint32_t M = 0x80000000u - C;
  const uint64_t p = (uint64_t)x * y;
  const uint64_t t = (p & 0x7FFFFFFFull) + (p >> 31) * C;
  const uint32_t r = (uint32_t)(t & 0x7FFFFFFFull) + (uint32_t)(t >> 31) * C;
  return umin32(r, r - M);
}

// a^e mod (2^31 - C) by square-and-multiply.
template <uint32_t C>
__device__ __forceinline__ uint32_t powmod_pm(uint32_t a, uint64_t e) {
  uint32_t r = 1, b = a;
  while (e) {
    if (e & 1) r = mulmod_pm<C>(r, b);
    b = mulmod_pm<C>(b, b);
    e >>= 1;
  }
  return r;
}

// Exact float of a u32 draw: (v >> SH) < 2^24 converts exactly, and the
// power-of-two scale is exact.
template <int SH>
__device__ __forceinline__ uint32_t as_f32_bits(uint32_t v) {
  return __float_as_uint(__uint2float_rn(v >> SH) * 0x1p-24f);
}

// Streaming store: outputs are written once and never read back here.
__device__ __forceinline__ void st_out(uint32_t* p, uint32_t v) { __stcs(p, v); }
__device__ __forceinline__ void st_out4(uint32_t* p, uint4 v) {
  __stcs(reinterpret_cast<uint4*>(p), v);
}

// Double of the consecutive draws a (high part) then b (reading R11), for
// generators whose words have WB significant bits: 24-bit words give
// m 2^-48 with m = a 2^24 + b; 31- and 32-bit words give m 2^-53 with m =
// (top 27 bits of a) 2^26 + (top 26 bits of b).  m has at most 53 bits, so
// the value is exact.  The bits are assembled with 32-bit integer
// instructions (the FP64 units of this GPU are slow): with the top bit of m
// at q, the fraction is m shifted left to put that bit at 52 (a funnel shift
// of its two words), and the exponent field 1022 + q - TOT is added to the
// high word, the fraction's own bit 52 completing it to 1023 + q - TOT.
// When the high part is zero (once in 2^24 or 2^27 pairs) a separate,
// never-inlined FP64 conversion takes over, so the common path stays free
// of FP64 instructions.
static __device__ __noinline__ double pair_f64_low_only(uint32_t lo, double scale) {
  return (double)lo * scale;
}

template <int WB>
__device__ __forceinline__ double pair_f64(uint32_t a, uint32_t b) {
  constexpr int LB = WB == 24 ? 24 : 26, TOT = WB == 24 ? 48 : 53;
  const uint32_t hi = WB == 24 ? a : a >> (WB - 27);
  const uint32_t lo = WB == 24 ? b : b >> (WB - 26);
  if (hi == 0) return pair_f64_low_only(lo, WB == 24 ? 0x1p-48 : 0x1p-53);
  const int z = __clz(hi);                          // q = 31 - z + LB
  const int s = 52 - (31 - z + LB);                 // 0 .. 28
  const uint32_t mh = hi >> (32 - LB), ml = (hi << LB) | lo;
  const uint32_t H = __funnelshift_l(ml, mh, s);    // high word of m << s
  const uint32_t L = ml << s;
  const uint32_t Hx = H + ((uint32_t)(1022 + 31 + LB - TOT - z) << 20);
  return __hiloint2double((int)Hx, (int)L);
}

// Stores of converted pairs at the u32 slot p of the pair's first draw
// (8-byte aligned: pairs start at even slots of 8-byte-aligned rows).
template <int WB>
__device__ __forceinline__ void st_pair(uint32_t* p, uint32_t a, uint32_t b) {
  __stcs(reinterpret_cast<double*>(p), pair_f64<WB>(a, b));
}
template <int WB>
__device__ __forceinline__ void st_pair4(uint32_t* p, uint4 v) {
  __stcs(reinterpret_cast<double2*>(p), make_double2(pair_f64<WB>(v.x, v.y), pair_f64<WB>(v.z, v.w)));
}

// A 16-byte chunk of four draws in output mode OM (pairs for OUT_F64).
template <int OM, int WB>
__device__ __forceinline__ void st_chunk(uint32_t* p, uint4 v) {
  if constexpr (OM == OUT_F64) st_pair4<WB>(p, v);
  else st_out4(p, v);
}

// Metropolis update of the site of colour rank k with draw v (the same rule
// as k_ising_half_sweep): accept when dE = 2 s (sum of neighbours) <= 0, or
// the 24-bit value v >> shift is below t4 (dE = 4) or t8 (dE = 8).  Sites of
// one colour only neighbour the other colour, so updates of one half-sweep
// never race.
__device__ __forceinline__ void ising_site(const IsingSink& q, uint32_t k, uint32_t v) {
  const uint32_t L = q.L, half = q.half;
  const uint32_t y = q.lg_half < 32 ? k >> q.lg_half : k / half;
  const uint32_t x = 2 * (k - y * half) + ((y + q.colour) & 1u);
  const uint32_t yu = y == 0 ? L - 1 : y - 1, yd = y + 1 == L ? 0 : y + 1;
  const uint32_t xl = x == 0 ? L - 1 : x - 1, xr = x + 1 == L ? 0 : x + 1;
  int8_t* row = q.spins + (uint64_t)y * L;
  const int s = row[x];
  const int nb = q.spins[(uint64_t)yu * L + x] + q.spins[(uint64_t)yd * L + x] + row[xl] + row[xr];
  const int dE = 2 * s * nb;
  const uint32_t r = v >> q.shift;
  if (dE <= 0 || (dE == 4 ? r < q.t4 : r < q.t8)) row[x] = (int8_t)(-s);
}

// The same update of the four sites of colour ranks k .. k+3, k % 4 == 0,
// with L % 8 == 0: they lie in one row at bytes xb .. xb+7 (xb = 2 (k - y L/2),
// a multiple of 8), every other byte, so the row chunk and the chunks above
// and below are single 8-byte loads, one byte beside the chunk completes the
// neighbours, and the chunk goes back as one 8-byte store.  The store also
// rewrites the chunk's other-colour bytes with the values it read; nothing
// changes them during the half-sweep.
__device__ __forceinline__ void ising_site4(const IsingSink& q, uint32_t k, uint4 v) {
  const uint32_t L = q.L, half = q.half;
  const uint32_t y = q.lg_half < 32 ? k >> q.lg_half : k / half;
  const uint32_t xb = 2 * (k - y * half);
  const uint32_t par = (y + q.colour) & 1u;
  const uint32_t yu = y == 0 ? L - 1 : y - 1, yd = y + 1 == L ? 0 : y + 1;
  int8_t* row = q.spins + (uint64_t)y * L;
  union B8 { uint2 v; int8_t c[8]; };
  B8 C, U, D;
  C.v = *reinterpret_cast<const uint2*>(row + xb);
  U.v = *reinterpret_cast<const uint2*>(q.spins + (uint64_t)yu * L + xb);
  D.v = *reinterpret_cast<const uint2*>(q.spins + (uint64_t)yd * L + xb);
  const int side = par ? row[xb + 8 == L ? 0 : xb + 8] : row[xb == 0 ? L - 1 : xb - 1];
  const uint32_t dr[4] = {v.x, v.y, v.z, v.w};
  B8 O = C;
#pragma unroll
  for (int i = 0; i < 4; i++) {
#pragma unroll
    for (int p = 0; p < 2; p++) {
      if ((uint32_t)p != par) continue;
      const int bi = 2 * i + p;
      const int s = C.c[bi];
      const int l = bi == 0 ? side : C.c[bi - 1];
      const int r = bi == 7 ? side : C.c[bi + 1];
      const int dE = 2 * s * (U.c[bi] + D.c[bi] + l + r);
      const uint32_t a = dr[i] >> q.shift;
      if (dE <= 0 || (dE == 4 ? a < q.t4 : a < q.t8)) O.c[bi] = (int8_t)(-s);
    }
  }
  *reinterpret_cast<uint2*>(row + xb) = O.v;
}

// Output of four consecutive draws (element index e of the first, at p) or
// of one: stored, or consumed by the fused half-sweep.
template <int OM, int WB>
__device__ __forceinline__ void put4(const FillDesc& d, uint32_t* p, uint64_t e, uint4 v) {
  if constexpr (OM == OUT_ISING) {
    if (d.ising.vec4 && (e & 3) == 0) {
      ising_site4(d.ising, (uint32_t)e, v);
    } else {
      ising_site(d.ising, (uint32_t)e, v.x);
      ising_site(d.ising, (uint32_t)e + 1, v.y);
      ising_site(d.ising, (uint32_t)e + 2, v.z);
      ising_site(d.ising, (uint32_t)e + 3, v.w);
    }
  } else {
    st_chunk<OM, WB>(p, v);
  }
}
template <int OM>
__device__ __forceinline__ void put1(const FillDesc& d, uint32_t* p, uint64_t e, uint32_t v) {
  if constexpr (OM == OUT_ISING) ising_site(d.ising, (uint32_t)e, v);
  else st_out(p, v);
}

// Row-major staging tile: thread t's staged draws in row t (SPW words per
// row, SPW = 4 mod 8 so that eight threads storing the same 16-byte chunk
// of their rows hit eight different bank quads).  RowFlusher writes tile
// columns [0, w) of rows row0 + t to out columns g0 .. g0 + w - 1.  Lanes
// take (row ro of a 4-row group, 16-byte chunk qq of an 8-chunk group) of
// the output, aligned to global multiples of 4 columns: when g0 is not a
// multiple of 4 a chunk straddles two tile chunks and is assembled from two
// 16-byte shared loads.  Eight lanes of a row read 128 contiguous bytes of
// shared memory, and a warp store covers 4 rows x 128 bytes of the output.
// LIMITED: honour FillDesc::limit (batched requests).  OM == OUT_F64: the
// staged words are raw draws of WB bits and each aligned pair (even global
// column, the next one) leaves as one double; g0, w and the limit are then
// even, so a pair is never split by a flush or a cut.
template <int T, int SPW, bool LIMITED = false, int OM = OUT_U32, int WB = 32>
struct RowFlusher {
  const FillDesc* dp;  // OUT_ISING: the sink
  uint64_t ebase;      // element index of this lane's first row, column 0
  const uint32_t* tile;              // OUT_ISING: the whole tile, rows row0 ..
  uint64_t irow0, ipitch, irows;     //   and their rows in the output
  static_assert(SPW % 8 == 4, "row pitch must be 4 mod 8 words");
  static constexpr int NW = T / 32, RIT = T / (4 * NW);
  uint32_t* gp;        // this lane's first row, column 0
  uint64_t rowstep;    // elements between this lane's rows
  const uint32_t* sp;  // tile row of this lane's first row
  int nrow, kcut, qq;
  uint64_t ccut;
  bool vec_ok;

  __device__ __forceinline__ void init(const uint32_t* s, uint32_t* out, uint64_t pitch,
                                       uint64_t row0, uint64_t n_rows, uint64_t limit,
                                       const FillDesc* d = nullptr) {
    // A quarter-warp (one 16-byte shared access phase) reads eight chunks of
    // one row: bank quads r * SPW / 4 + chunk (mod 8), all different.
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int r = wi * 4 + (lane >> 3);
    qq = lane & 7;
    rowstep = (uint64_t)NW * 4 * pitch;
    dp = d;
    ebase = (row0 + r) * pitch;
    tile = s;
    irow0 = row0;
    ipitch = pitch;
    irows = n_rows;
    gp = out + (row0 + r) * pitch;
    sp = s + r * SPW;
    uint64_t rows = n_rows;
    if (LIMITED && pitch > 0 && (limit + pitch - 1) / pitch < rows) rows = (limit + pitch - 1) / pitch;
    const uint64_t left = rows > row0 + r ? rows - (row0 + r) : 0;
    const uint64_t nr = (left + (NW * 4 - 1)) / (NW * 4);
    nrow = nr < (uint64_t)RIT ? (int)nr : RIT;
    kcut = RIT;
    ccut = 0;
    if (LIMITED && pitch > 0 && limit < rows * pitch) {
      const uint64_t last = rows - 1;
      if (last >= row0 + r && (last - (row0 + r)) % (NW * 4) == 0) {
        kcut = (int)((last - (row0 + r)) / (NW * 4));
        ccut = limit - last * pitch;
      }
    }
    vec_ok = ((pitch & 3) == 0) && ((reinterpret_cast<uintptr_t>(out) & 15) == 0);
  }

  template <int A>
  __device__ __forceinline__ void flush_a(uint64_t g0, int w) const {
    const uint64_t q0 = g0 >> 2;
    const int nq = (int)(((g0 + (uint64_t)w + 3) >> 2) - q0);
    for (int qb = 0; qb < nq; qb += 8) {
      const int qi = qb + qq;
      if (qi >= nq) continue;
      const uint64_t gc = (q0 + qi) * 4;
      const int c = (int)(gc - g0);           // tile column of the chunk's first element
      uint32_t* g = gp + gc;
      const bool full = vec_ok && c >= 0 && c + 4 <= w;
      const uint32_t* t = sp + (c - A);       // 16-byte aligned: c = A (mod 4)
#pragma unroll
      for (int k = 0; k < RIT; k++) {
        if (k >= nrow) break;
        const uint32_t* tk = t + k * NW * 4 * SPW;
        uint32_t v[4];
        if (full) {
          const uint4 lo = *reinterpret_cast<const uint4*>(tk);
          if constexpr (A == 0) {
            v[0] = lo.x; v[1] = lo.y; v[2] = lo.z; v[3] = lo.w;
          } else {
            const uint4 hi = *reinterpret_cast<const uint4*>(tk + 4);
            const uint32_t u[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
            for (int i = 0; i < 4; i++) v[i] = u[A + i];
          }
          if (!LIMITED || k != kcut || gc + 4 <= ccut) {
            if constexpr (OM == OUT_ISING)
              put4<OM, WB>(*dp, nullptr, ebase + gc + k * rowstep, make_uint4(v[0], v[1], v[2], v[3]));
            else
              st_chunk<OM, WB>(g + k * rowstep, make_uint4(v[0], v[1], v[2], v[3]));
            continue;
          }
        }
        if constexpr (OM == OUT_F64) {
#pragma unroll
          for (int i = 0; i < 4; i += 2) {
            const int ci = c + i;
            if (ci >= 0 && ci < w && (!LIMITED || k != kcut || gc + i < ccut))
              st_pair<WB>(g + k * rowstep + i, sp[k * NW * 4 * SPW + ci], sp[k * NW * 4 * SPW + ci + 1]);
          }
        } else {
#pragma unroll
          for (int i = 0; i < 4; i++) {
            const int ci = c + i;
            if (ci >= 0 && ci < w && (!LIMITED || k != kcut || gc + i < ccut)) {
              if constexpr (OM == OUT_ISING)
                ising_site(dp->ising, (uint32_t)(ebase + gc + k * rowstep + i), sp[k * NW * 4 * SPW + ci]);
              else
                st_out(g + k * rowstep + i, sp[k * NW * 4 * SPW + ci]);
            }
          }
        }
      }
    }
  }

  __device__ __forceinline__ void flush(uint64_t g0, int w) const {
    if constexpr (OM == OUT_ISING) {
      // The fused half-sweep: every staged draw updates its site.  The
      // CTA's threads take the tile's elements in row order, four at a time
      // (consecutive threads, consecutive quads of colour ranks: one 8-byte
      // chunk of a lattice row each when the ranks are 4-aligned), stepping
      // (row, quad) by T quads without a division per quad; the columns
      // past the last whole quad go one at a time.
      const int wq = w >> 2;
      if (wq > 0) {
        const int qT = T / wq, rT = T - qT * wq;
        int r = threadIdx.x / wq, c = threadIdx.x - r * wq;
        for (int i = threadIdx.x; i < T * wq; i += T) {
          if (irow0 + r < irows) {
            const uint32_t e = (uint32_t)((irow0 + r) * ipitch + g0) + (uint32_t)(4 * c);
            const uint32_t* t = tile + r * SPW + 4 * c;
            put4<OUT_ISING, WB>(*dp, nullptr, e, make_uint4(t[0], t[1], t[2], t[3]));
          }
          r += qT;
          c += rT;
          if (c >= wq) {
            c -= wq;
            r++;
          }
        }
      }
      const int wr = w - 4 * wq;
      for (int i = threadIdx.x; i < T * wr; i += T) {
        const int r = i / wr, c = 4 * wq + (i - r * wr);
        if (irow0 + r < irows)
          ising_site(dp->ising, (uint32_t)((irow0 + r) * ipitch + g0) + (uint32_t)c, tile[r * SPW + c]);
      }
    } else {
      switch ((uint32_t)(0u - (uint32_t)g0) & 3u) {
        case 0: flush_a<0>(g0, w); break;
        case 2: flush_a<2>(g0, w); break;
        case 1: if constexpr (OM != OUT_F64) flush_a<1>(g0, w); break;
        default: if constexpr (OM != OUT_F64) flush_a<3>(g0, w); break;
      }
    }
  }
};

}  // namespace prng
