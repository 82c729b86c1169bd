// k_ranlux.cu -- RANLUX fill and skip (Section 3.6; Appendix A, "AWC and SWB"
// and "RANLUX").
//
// One thread per stream.  The 24-word RCARRY ring and the borrow live in
// registers: the ring is walked 24 steps at a time with compile-time phase,
// so every lag index (x_{n-10}, x_{n-24}) is a fixed register.  A luxury
// cycle is 24 delivered steps plus p - 24 discarded ones; p - 24 = 24 q + r
// runs as q unrolled 24-step groups, r single steps and one fixed register
// permutation that re-aligns the ring.  Runtime-length pieces (the head of a
// fill that resumes mid-block, the tail of a short fill) take guarded steps
// followed by a barrel rotation (5 conditional fixed permutations).
//
// Delivered values are staged per thread into a shared-memory row (odd row
// pitch: conflict-free scalar stores) and written out row by row when the
// tile is full, which makes the stream-major HBM writes contiguous.
#include "common.cuh"

namespace prng {

// One SWB step at compile-time ring phase k: V[j] = R[(j + k) % 24],
// x_n = (x_{n-10} - x_{n-24} - c) mod 2^24, c = borrow.
__device__ __forceinline__ void swb_step(uint32_t (&R)[24], uint32_t& c, const int k) {
  const int i0 = k % 24, i14 = (k + 14) % 24;
  const int32_t t = (int32_t)R[i14] - (int32_t)R[i0] - (int32_t)c;
  c = (uint32_t)t >> 31;
  R[i0] = (uint32_t)t & 0xFFFFFFu;
}

// Re-align after s steps: new R[j] = R[(j + s) % 24] (s a compile-time value).
__device__ __forceinline__ void rotate_fixed(uint32_t (&R)[24], const int s) {
  uint32_t tmp[24];
#pragma unroll
  for (int j = 0; j < 24; j++) tmp[j] = R[(j + s) % 24];
#pragma unroll
  for (int j = 0; j < 24; j++) R[j] = tmp[j];
}

// Re-align after a runtime number of steps h in [0, 24).
__device__ __forceinline__ void rotate_runtime(uint32_t (&R)[24], int h) {
  if (h & 1) rotate_fixed(R, 1);
  if (h & 2) rotate_fixed(R, 2);
  if (h & 4) rotate_fixed(R, 4);
  if (h & 8) rotate_fixed(R, 8);
  if (h & 16) rotate_fixed(R, 16);
}

template <bool F32>
__device__ __forceinline__ uint32_t lux_conv(uint32_t x) {
  if constexpr (F32) return __float_as_uint(__uint2float_rn(x) * 0x1p-24f);
  else return x;
}

// p - 24 discarded steps; leaves the ring at phase 0.
template <int P>
__device__ __forceinline__ void discard_cycle(uint32_t (&R)[24], uint32_t& c) {
  constexpr int D = P - 24, Q = D / 24, RR = D % 24;
  for (int g = 0; g < Q; g++) {
#pragma unroll
    for (int k = 0; k < 24; k++) swb_step(R, c, k);
  }
#pragma unroll
  for (int k = 0; k < RR; k++) swb_step(R, c, k);
  if constexpr (RR != 0) rotate_fixed(R, RR);
}

template <int T, int KT, int P, bool F32>
__global__ void __launch_bounds__(T) k_fill_ranlux(const FillDesc d) {
  constexpr int SP = KT + 1;  // odd pitch: a warp's scalar stores hit 32 banks
  extern __shared__ uint32_t smem[];
  const int tid = threadIdx.x;
  const uint64_t row0 = (uint64_t)blockIdx.x * T;
  const uint64_t row = row0 + tid;
  const bool active = row < d.n_rows;
  const uint64_t nr = d.n_rows;

  uint32_t R[24];
  uint32_t c = 0;
  if (active) {
#pragma unroll
    for (int j = 0; j < 24; j++) R[j] = d.state[j * nr + row];
    c = d.state[24 * nr + row];
  } else {
#pragma unroll
    for (int j = 0; j < 24; j++) R[j] = 0;
  }

  uint32_t* out = static_cast<uint32_t*>(d.out);
  const bool store = out != nullptr;
  uint32_t* my = smem + tid * SP;
  int fill = 0;        // staged columns (uniform)
  uint64_t g0 = 0;     // output column of staged column 0

  auto flush = [&]() {
    __syncthreads();
    copy_rows_scalar<T>(smem, SP, out, d.pitch, row0, nr, g0, fill, d.limit);
    __syncthreads();
    g0 += fill;
    fill = 0;
  };

  // Deliver h (< 24, runtime) steps at phase 0, then re-align.
  auto deliver_partial = [&](int h) {
    if (store && fill + h > KT) flush();
#pragma unroll
    for (int k = 0; k < 24; k++) {
      if (k < h) {
        swb_step(R, c, k);
        if (store) my[fill + k] = lux_conv<F32>(R[k]);
      }
    }
    fill += h;
    rotate_runtime(R, h);
  };

  const uint64_t n = d.n_per;
  uint64_t j = 0;
  int pos = (int)d.pos;
  if (pos < 24 && n > 0) {  // finish the block a previous call left open
    const int h = (int)((uint64_t)(24 - pos) < n ? (uint64_t)(24 - pos) : n);
    deliver_partial(h);
    j += h;
  }
  while (j < n) {  // the open block is complete here: discard, then deliver
    discard_cycle<P>(R, c);
    if (n - j >= 24) {
      if (store && fill + 24 > KT) flush();
#pragma unroll
      for (int k = 0; k < 24; k++) {
        swb_step(R, c, k);
        if (store) my[fill + k] = lux_conv<F32>(R[k]);
      }
      fill += 24;
      j += 24;
    } else {
      const int h = (int)(n - j);
      deliver_partial(h);
      j += h;
    }
  }
  if (store && fill > 0) flush();

  if (active) {
#pragma unroll
    for (int jj = 0; jj < 24; jj++) d.state[jj * nr + row] = R[jj];
    d.state[24 * nr + row] = c;
  }
}

template <int T, int KT, int P, bool F32>
static cudaError_t launch_l(const FillDesc& d, cudaStream_t s) {
  constexpr size_t bytes = (size_t)T * (KT + 1) * sizeof(uint32_t);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_fill_ranlux<T, KT, P, F32>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const uint64_t grid = (d.n_rows + T - 1) / T;
  k_fill_ranlux<T, KT, P, F32><<<(unsigned)grid, T, d.out ? bytes : 0, s>>>(d);
  return cudaGetLastError();
}

template <int T, int KT, int P>
static cudaError_t launch_lp(const FillDesc& d, cudaStream_t s) {
  return d.f32 ? launch_l<T, KT, P, true>(d, s) : launch_l<T, KT, P, false>(d, s);
}

template <int T, int KT>
static cudaError_t launch_lt(const FillDesc& d, cudaStream_t s) {
  switch (d.p) {
    case 24: return launch_lp<T, KT, 24>(d, s);
    case 48: return launch_lp<T, KT, 48>(d, s);
    case 97: return launch_lp<T, KT, 97>(d, s);
    case 223: return launch_lp<T, KT, 223>(d, s);
    case 389: return launch_lp<T, KT, 389>(d, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_fill_ranlux(const FillDesc& d, Tile t, cudaStream_t s) {
  if (d.n_rows == 0 || d.n_per == 0) return cudaSuccess;
  if (t.threads == 64) return launch_lt<64, 48>(d, s);
  return launch_lt<128, 48>(d, s);
}

}  // namespace prng
