// k_ranmar.cu -- RANMAR fill and skip (Section 3.5; Appendix A, "RANMAR").
//
// One thread per stream with the whole 97-entry lag table in registers.
// The two table indices (i97, j97) fall together by one per draw and are
// the same for every stream, so the state is kept in canonical order
// (V[0] = the entry overwritten next) and the kernel walks the table 97
// draws at a time with compile-time phase: entry k of the unrolled block
// reads registers k and (k + 64) mod 97 and writes register k.  A fill of n
// draws runs n / 97 full blocks and one guarded partial block; the final
// phase is folded into the store-back addresses, so no register is ever
// indexed at run time.  The Weyl term C_n = C_{n-1} - D mod M is a short
// side chain.  Each block's 97 draws are staged in a shared-memory row and
// written out row by row.
#include "common.cuh"

namespace prng {

constexpr uint32_t kRanmarD = 7654321u;    // Section 3.5: RM_CD * 2^24
constexpr uint32_t kRanmarM = 16777213u;   // Section 3.5: RM_CM * 2^24

// Draw at compile-time phase k: Y = V[0] - V[64] mod 2^24 replaces V[0];
// C <- C - D (+M when negative); X = Y - C mod 2^24.
__device__ __forceinline__ uint32_t ranmar_step(uint32_t (&R)[97], uint32_t& C, const int k) {
  const int i0 = k % 97, i64 = (k + 64) % 97;
  const uint32_t y = (R[i0] - R[i64]) & 0xFFFFFFu;
  R[i0] = y;
  C -= kRanmarD;
  C += ((int32_t)C < 0) ? kRanmarM : 0u;
  return (y - C) & 0xFFFFFFu;
}

template <bool F32>
__device__ __forceinline__ uint32_t rm_conv(uint32_t x) {
  if constexpr (F32) return __float_as_uint(__uint2float_rn(x) * 0x1p-24f);
  else return x;
}

template <int T, bool F32>
__global__ void __launch_bounds__(T) k_fill_ranmar(const FillDesc d) {
  constexpr int KT = 97, SP = 97;  // one block per tile; odd pitch
  extern __shared__ uint32_t smem[];
  const int tid = threadIdx.x;
  const uint64_t row0 = (uint64_t)blockIdx.x * T;
  const uint64_t row = row0 + tid;
  const bool active = row < d.n_rows;
  const uint64_t nr = d.n_rows;

  uint32_t R[97];
  uint32_t C = 0;
  if (active) {
#pragma unroll
    for (int j = 0; j < 97; j++) R[j] = d.state[j * nr + row];
    C = d.state[97 * nr + row];
  } else {
#pragma unroll
    for (int j = 0; j < 97; j++) R[j] = 0;
  }

  uint32_t* out = static_cast<uint32_t*>(d.out);
  const bool store = out != nullptr;
  uint32_t* my = smem + tid * SP;
  const uint64_t n = d.n_per;
  const uint64_t nfull = n / 97;
  const int m = (int)(n % 97);
  uint64_t g0 = 0;

  for (uint64_t b = 0; b < nfull; b++) {
#pragma unroll
    for (int k = 0; k < 97; k++) {
      const uint32_t x = ranmar_step(R, C, k);
      if (store) my[k] = rm_conv<F32>(x);
    }
    if (store) {
      __syncthreads();
      copy_rows_scalar<T>(smem, SP, out, d.pitch, row0, nr, g0, KT, d.limit);
      __syncthreads();
    }
    g0 += KT;
  }
  if (m > 0) {
#pragma unroll
    for (int k = 0; k < 97; k++) {
      if (k < m) {
        const uint32_t x = ranmar_step(R, C, k);
        if (store) my[k] = rm_conv<F32>(x);
      }
    }
    if (store) {
      __syncthreads();
      copy_rows_scalar<T>(smem, SP, out, d.pitch, row0, nr, g0, m, d.limit);
    }
  }

  if (active) {
    // After n draws the ring phase is m: canonical V[k] = R[(k + m) % 97].
#pragma unroll
    for (int r = 0; r < 97; r++) {
      const int k = (r - m + 97) % 97;
      d.state[(uint64_t)k * nr + row] = R[r];
    }
    d.state[97 * nr + row] = C;
  }
}

template <int T, bool F32>
static cudaError_t launch_m(const FillDesc& d, cudaStream_t s) {
  constexpr size_t bytes = (size_t)T * 97 * sizeof(uint32_t);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_fill_ranmar<T, F32>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const uint64_t grid = (d.n_rows + T - 1) / T;
  k_fill_ranmar<T, F32><<<(unsigned)grid, T, d.out ? bytes : 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_fill_ranmar(const FillDesc& d, Tile t, cudaStream_t s) {
  if (d.n_rows == 0 || d.n_per == 0) return cudaSuccess;
  if (t.threads == 128) return d.f32 ? launch_m<128, true>(d, s) : launch_m<128, false>(d, s);
  return d.f32 ? launch_m<64, true>(d, s) : launch_m<64, false>(d, s);
}

}  // namespace prng
