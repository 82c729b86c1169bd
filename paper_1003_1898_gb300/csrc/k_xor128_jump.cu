// k_xor128_jump.cu -- XOR128 jump-ahead over GF(2) (Appendix A, "XORShift",
// matrix form).
//
// The XOR128 state (x, y, z, w) is a vector of 128 bits (bit 32 i + b is bit
// b of word i, words in the order x, y, z, w), and one step multiplies it
// by a 128 x 128 matrix T over GF(2).  k steps multiply by T^k, which the
// host forms as the product of the powers T^(2^b) for the set bits b of k
// (the 64 powers are squared out once per process and kept), each matrix
// kept as its 128 columns of four words.  The device applies
// a matrix to many states at once: the image of v is the XOR of the columns
// selected by v's set bits, with the matrix passed by value in the launch
// parameters (2 KB), read by every thread at the same address.
//
//  * prng_skip on an XOR128 handle: T^k applied to every stream's state.
//  * The single-sequence fill from x0: chunk c of L draws starts from
//    T^(cL) s0 (chunks are cut finer than asked when there are too few to
//    fill the GPU).  The chunk starts are built in log8(C) passes of three
//    doubling levels each (starts [H, 8H) from starts [0, H) by products of
//    the powers T^(L H), T^(2 L H), T^(4 L H)) in a stream-ordered scratch
//    array, then the ordinary XOR128 fill kernel runs with one chunk per row.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "scratch.cuh"

namespace prng {

struct Gf2x128 {
  uint32_t col[128][4];   // col[j] = T e_j
};

// Chunks the single-sequence fill uses at least (when the sequence is long
// enough): one thread each, as many as the bulk XOR128 fill keeps resident.
constexpr uint64_t kJumpRows = 131072;

namespace {

// One XOR128 step on a host-side state (Appendix A, "XORShift", scalar form).
void xs_step(uint32_t v[4]) {
  const uint32_t t = v[0] ^ (v[0] << 11);
  v[0] = v[1];
  v[1] = v[2];
  v[2] = v[3];
  v[3] = (v[3] ^ (v[3] >> 19)) ^ (t ^ (t >> 8));
}

void gf2_apply(const Gf2x128& A, const uint32_t v[4], uint32_t out[4]) {
  uint32_t r0 = 0, r1 = 0, r2 = 0, r3 = 0;
  for (int j = 0; j < 128; j++) {
    if ((v[j >> 5] >> (j & 31)) & 1u) {
      r0 ^= A.col[j][0];
      r1 ^= A.col[j][1];
      r2 ^= A.col[j][2];
      r3 ^= A.col[j][3];
    }
  }
  out[0] = r0; out[1] = r1; out[2] = r2; out[3] = r3;
}

// C = A B (C may alias A or B).
void gf2_mul(const Gf2x128& A, const Gf2x128& B, Gf2x128& C) {
  Gf2x128 t;
  for (int j = 0; j < 128; j++) gf2_apply(A, B.col[j], t.col[j]);
  C = t;
}

Gf2x128 gf2_identity() {
  Gf2x128 I{};
  for (int j = 0; j < 128; j++) I.col[j][j >> 5] = 1u << (j & 31);
  return I;
}

Gf2x128 xor128_step_matrix() {
  Gf2x128 T{};
  for (int j = 0; j < 128; j++) {
    uint32_t v[4] = {0, 0, 0, 0};
    v[j >> 5] = 1u << (j & 31);
    xs_step(v);
    for (int i = 0; i < 4; i++) T.col[j][i] = v[i];
  }
  return T;
}

// T^(2^i) for i < 64, formed once by repeated squaring (128 KB).
const Gf2x128* pow2_table() {
  static Gf2x128 table[64];
  static std::once_flag once;
  std::call_once(once, [] {
    table[0] = xor128_step_matrix();
    for (int i = 1; i < 64; i++) gf2_mul(table[i - 1], table[i - 1], table[i]);
  });
  return table;
}

// T^(k 2^shift) = product of T^(2^(b + shift)) over the set bits b of k
// (k 2^shift < 2^64).
Gf2x128 step_power(uint64_t k, int shift = 0) {
  const Gf2x128* P = pow2_table();
  Gf2x128 R = gf2_identity();
  bool first = true;
  for (int b = 0; b + shift < 64 && (k >> b) != 0; b++) {
    if (!((k >> b) & 1)) continue;
    if (first) R = P[b + shift];
    else gf2_mul(P[b + shift], R, R);
    first = false;
  }
  return R;
}

}  // namespace

// x = M x on the device, M passed in the launch parameters.  Fully unrolled
// over the 128 bits of x, so that every column word is a constant-bank
// operand of its XOR and the state stays in registers.
__device__ __forceinline__ void gf2_apply_dev(const Gf2x128& M, uint32_t x[4]) {
  uint32_t o0 = 0, o1 = 0, o2 = 0, o3 = 0;
#pragma unroll
  for (int w = 0; w < 4; w++) {
    const uint32_t xw = x[w];
#pragma unroll
    for (int b = 0; b < 32; b++) {
      const uint32_t m = 0u - ((xw >> b) & 1u);
      o0 ^= M.col[32 * w + b][0] & m;
      o1 ^= M.col[32 * w + b][1] & m;
      o2 ^= M.col[32 * w + b][2] & m;
      o3 ^= M.col[32 * w + b][3] & m;
    }
  }
  x[0] = o0; x[1] = o1; x[2] = o2; x[3] = o3;
}

// Rows [r0, r1) of a struct-of-arrays XOR128 state (pitch rows per word)
// become M times row (r - src_off).  With src_off = 0 the update is in place
// (each thread reads its row before writing it).
__global__ void __launch_bounds__(256) k_xor128_apply(const __grid_constant__ Gf2x128 M,
                                                      uint32_t* state, uint64_t pitch, uint64_t r0,
                                                      uint64_t r1, uint64_t src_off) {
  const uint64_t r = r0 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= r1) return;
  const uint64_t src = r - src_off;
  uint32_t x[4];
#pragma unroll
  for (int i = 0; i < 4; i++) x[i] = state[i * pitch + src];
  gf2_apply_dev(M, x);
#pragma unroll
  for (int i = 0; i < 4; i++) state[i * pitch + r] = x[i];
}

struct Gf2x128x3 {
  Gf2x128 m[3];   // T^E, T^(2E), T^(4E)
};

// Three doubling levels in one pass: with the chunk starts [0, H) known,
// chunk r = j H + s (j = 1..7, s < H) starts at T^(j E) applied to start
// s, E = L H the draws of H chunks.  One thread per r < C applies the
// powers T^E, T^(2E), T^(4E) picked by the bits of j (at most three
// products), so the host multiplies no matrices and a pass is one launch.
__global__ void __launch_bounds__(256) k_xor128_apply3(const __grid_constant__ Gf2x128x3 P,
                                                       uint32_t* state, uint64_t pitch,
                                                       uint64_t H, uint64_t C) {
  const uint64_t r = H + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= C || r >= 8 * H) return;
  const uint64_t j = r / H, s = r - j * H;
  uint32_t x[4];
#pragma unroll
  for (int i = 0; i < 4; i++) x[i] = state[i * pitch + s];
  if (j & 4) gf2_apply_dev(P.m[2], x);
  if (j & 2) gf2_apply_dev(P.m[1], x);
  if (j & 1) gf2_apply_dev(P.m[0], x);
#pragma unroll
  for (int i = 0; i < 4; i++) state[i * pitch + r] = x[i];
}

__global__ void k_xor128_set_row(uint32_t* state, uint64_t pitch, uint64_t row, uint32_t x,
                                 uint32_t y, uint32_t z, uint32_t w) {
  state[row] = x;
  state[pitch + row] = y;
  state[2 * pitch + row] = z;
  state[3 * pitch + row] = w;
}

static cudaError_t apply_rows(const Gf2x128& M, uint32_t* state, uint64_t pitch, uint64_t r0,
                              uint64_t r1, uint64_t src_off, cudaStream_t s) {
  if (r1 <= r0) return cudaSuccess;
  const uint64_t blocks = (r1 - r0 + 255) / 256;
  if (blocks > 0x7FFFFFFFull) return cudaErrorInvalidValue;
  k_xor128_apply<<<(unsigned)blocks, 256, 0, s>>>(M, state, pitch, r0, r1, src_off);
  return cudaGetLastError();
}

cudaError_t launch_skip_xor128(uint32_t* state, uint64_t n, uint64_t k, cudaStream_t s) {
  if (n == 0 || k == 0) return cudaSuccess;
  const Gf2x128 M = step_power(k);
  return apply_rows(M, state, n, 0, n, 0, s);
}

cudaError_t launch_jump_xor128(uint64_t x0, uint64_t first, uint64_t n, uint32_t n_chunks,
                               void* d_out, int f32, cudaStream_t s) {
  // The fill kernel runs one thread per chunk, so the chunks are cut finer
  // when there are too few to fill the GPU (any contiguous cut of the one
  // sequence gives the same output), down to 64 draws per chunk.
  const uint64_t want = std::max<uint64_t>(n_chunks, std::min<uint64_t>((n + 63) / 64, kJumpRows));
  const uint64_t L = (n + want - 1) / want;           // draws per chunk
  const uint64_t C = (n + L - 1) / L;                 // chunks, none empty
  // Start state: the stream seeding map for the per-stream value s = x0.
  const uint64_t t = splitmix64(x0);
  uint32_t v0[4] = {(uint32_t)x0, (uint32_t)(x0 >> 32), (uint32_t)t, (uint32_t)(t >> 32)};
  if ((v0[0] | v0[1] | v0[2] | v0[3]) == 0) v0[3] = 1;

  uint32_t* S = nullptr;
  cudaError_t e = scratch_alloc(reinterpret_cast<void**>(&S), 4 * C * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  k_xor128_set_row<<<1, 1, 0, s>>>(S, C, 0, v0[0], v0[1], v0[2], v0[3]);
  e = cudaGetLastError();
  if (e == cudaSuccess && first > 0) e = apply_rows(step_power(first), S, C, 0, 1, 0, s);  // to `first`
  // Pass i: chunks [H, 8H) from chunks [0, H), H = 8^i, by T^(j L H).
  int i = 0;
  for (uint64_t H = 1; e == cudaSuccess && H < C; H <<= 3, i += 3) {
    Gf2x128x3 P;
    P.m[0] = step_power(L, i);
    P.m[1] = step_power(L, i + 1);
    P.m[2] = step_power(L, i + 2);
    const uint64_t rows = std::min<uint64_t>(C, 8 * H) - H;
    const uint64_t blocks = (rows + 255) / 256;
    if (blocks > 0x7FFFFFFFull) {
      e = cudaErrorInvalidValue;
      break;
    }
    k_xor128_apply3<<<(unsigned)blocks, 256, 0, s>>>(P, S, C, H, C);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    FillDesc d{};
    d.state = S;
    d.n_rows = C;
    d.n_per = L;
    d.out = d_out;
    d.pitch = L;
    d.limit = n;
    d.mode = f32 ? OUT_F32 : OUT_U32;
    e = launch_fill_simple(XOR128, d, default_tile(XOR128, 0), s);
  }
  const cudaError_t ef = scratch_free(S, s);
  return e != cudaSuccess ? e : ef;
}

}  // namespace prng
