// k_calib.cu -- measurement aid for the RANLUX roofline (no counterpart in
// the paper): the integer rate of the subtract-with-borrow chain that the
// RANLUX kernels run (Appendix A, "AWC and SWB": x_n = x_{n-10} - x_{n-24} -
// c), measured on the GPU at hand instead of assumed.
//
// Each thread holds CH independent 24-word rings and runs the RANLUX
// kernels' own 24-step chain (swb24: 24 subtract-with-borrow and 24
// low-byte clears, and 3 instructions to move the borrow in and out of the
// carry flag) on each of them, `iters` times.  With several rings per
// thread and every warp slot filled, the chains' latency is hidden and the
// launch runs at the integer pipe's throughput for this instruction mix;
// with one ring per thread and one warp per scheduler it runs at the
// chain's latency.
#include "../../include/prng.h"
#include "ranlux.cuh"

namespace prng {

template <int CH>
__global__ void __launch_bounds__(128) k_calib_swb(uint32_t iters, uint32_t* sink) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t R[CH][24], c[CH];
#pragma unroll
  for (int h = 0; h < CH; h++) {
    uint32_t x = tid * 2654435761u + 97u * h + 1u;
#pragma unroll
    for (int j = 0; j < 24; j++) {
      x = x * 1664525u + 1013904223u;
      R[h][j] = x & 0xFFFFFF00u;
    }
    c[h] = 0;
  }
  for (uint32_t i = 0; i < iters; i++) {
#pragma unroll
    for (int h = 0; h < CH; h++) swb24(R[h], c[h]);
  }
  uint32_t acc = 0;
#pragma unroll
  for (int h = 0; h < CH; h++) {
    acc += c[h];
#pragma unroll
    for (int j = 0; j < 24; j++) acc ^= R[h][j];
  }
  sink[tid] = acc;
}

template <int CH>
static cudaError_t calib_launch(uint32_t warps_per_sm, uint32_t iters, uint32_t* sink,
                                uint64_t sink_words, uint64_t* ops, cudaStream_t s) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_calib_swb<CH>, 128, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  // 128-thread blocks: warps_per_sm / 4 blocks per SM, at most what fits
  // at once, so that the launch is one wave.
  uint32_t blocks_per_sm = warps_per_sm == 0 ? (uint32_t)per_sm : (warps_per_sm + 3) / 4;
  if (blocks_per_sm > (uint32_t)per_sm) blocks_per_sm = (uint32_t)per_sm;
  const uint64_t grid = (uint64_t)sm_count() * blocks_per_sm;
  if (grid * 128 > sink_words) return cudaErrorInvalidValue;
  k_calib_swb<CH><<<(unsigned)grid, 128, 0, s>>>(iters, sink);
  *ops = grid * 128 * (uint64_t)CH * iters * (24 * 2 + 3);
  return cudaGetLastError();
}

}  // namespace prng

extern "C" int prng_calib_swb(uint32_t chains, uint32_t warps_per_sm, uint32_t iters,
                              uint32_t* d_sink, uint64_t sink_words, uint64_t* ops,
                              void* stream) {
  using namespace prng;
  if (d_sink == nullptr || ops == nullptr) return PRNG_ENULL;
  if (iters == 0) return PRNG_ESIZE;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  switch (chains) {
    case 1: e = calib_launch<1>(warps_per_sm, iters, d_sink, sink_words, ops, s); break;
    case 2: e = calib_launch<2>(warps_per_sm, iters, d_sink, sink_words, ops, s); break;
    case 4: e = calib_launch<4>(warps_per_sm, iters, d_sink, sink_words, ops, s); break;
    default: return PRNG_ESIZE;
  }
  if (e == cudaErrorInvalidValue) return PRNG_ESIZE;
  return e == cudaSuccess ? PRNG_OK : PRNG_ECUDA;
}
