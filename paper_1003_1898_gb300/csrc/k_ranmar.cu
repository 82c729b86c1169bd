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
// indexed at run time.  The Weyl term C_n = C_{n-1} - D mod M is evaluated
// per draw as an offset of the block's entry value by a compile-time
// constant, so no draw waits on the previous one.  Each block's 97 draws are staged in a column-major shared
// tile and written out 16 bytes at a time (ColFlusher).
#include "batch.cuh"

namespace prng {

constexpr uint32_t kRanmarD = 7654321u;    // Section 3.5: RM_CD * 2^24
constexpr uint32_t kRanmarM = 16777213u;   // Section 3.5: RM_CM * 2^24

// (k D) mod M, D = 7654321, M = 2^24 - 3 (a compile-time constant for the
// unrolled steps).
__host__ __device__ constexpr uint32_t ranmar_kd(int k) {
  return (uint32_t)(((uint64_t)k * kRanmarD) % kRanmarM);
}

// Draw k (compile-time, 0-based) of a block whose Weyl term entered the
// block as C0.  Y = V[0] - V[64] replaces V[0] (kept modulo 2^32; only its
// low 24 bits matter).  The Weyl term after k+1 steps is C0 - (k+1) D mod M,
// so each draw's C is an offset by a constant, independent of the previous
// draw: with c = C0 - ((k+1) D mod M), C = c when c >= 0 and c + M otherwise,
// and since M = 2^24 - 3, X = (Y - C) mod 2^24 = (Y - c + 3 [c < 0]) mod 2^24.
__device__ __forceinline__ uint32_t ranmar_step(uint32_t (&R)[97], uint32_t C0, const int k) {
  const int i0 = k % 97, i64 = (k + 64) % 97;
  const uint32_t y = R[i0] - R[i64];
  R[i0] = y;
  const int32_t c = (int32_t)C0 - (int32_t)ranmar_kd(k + 1);
  return (y - (uint32_t)c + 3u * ((uint32_t)c >> 31)) & 0xFFFFFFu;
}

// C0 after `steps` more draws.
__device__ __forceinline__ uint32_t ranmar_advance_c(uint32_t C0, uint32_t steps) {
  const uint32_t kd = (uint32_t)(((uint64_t)steps * kRanmarD) % kRanmarM);
  const int32_t c = (int32_t)C0 - (int32_t)kd;
  return c < 0 ? (uint32_t)(c + (int32_t)kRanmarM) : (uint32_t)c;
}

template <bool F32>
__device__ __forceinline__ uint32_t rm_conv(uint32_t x) {
  if constexpr (F32) return __float_as_uint(__uint2float_rn(x) * 0x1p-24f);
  else return x;
}

// Streams [row0, row0 + T) of a fill, one per thread; smem holds one
// column-major tile of 97 columns (see ColFlusher).
template <int T, bool F32, bool LIMITED>
__device__ __forceinline__ void ranmar_rows(const FillDesc& d, uint64_t row0, uint32_t* smem) {
  constexpr int SP = T + 1;
  const int tid = threadIdx.x;
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
  ColFlusher<T, LIMITED> fl;
  fl.init(smem, out, d.pitch, row0, nr, d.limit);
  uint32_t* col = smem + tid;
  const uint64_t n = d.n_per;
  const uint64_t nfull = n / 97;
  const int m = (int)(n % 97);
  uint64_t g0 = 0;

  for (uint64_t b = 0; b < nfull; b++) {
#pragma unroll
    for (int k = 0; k < 97; k++) {
      const uint32_t x = ranmar_step(R, C, k);
      if (store) col[k * SP] = rm_conv<F32>(x);
    }
    C = ranmar_advance_c(C, 97);
    if (store) {
      __syncthreads();
      fl.flush(g0, 97);
      __syncthreads();
    }
    g0 += 97;
  }
  if (m > 0) {
#pragma unroll
    for (int k = 0; k < 97; k++) {
      if (k < m) {
        const uint32_t x = ranmar_step(R, C, k);
        if (store) col[k * SP] = rm_conv<F32>(x);
      }
    }
    C = ranmar_advance_c(C, (uint32_t)m);
    if (store) {
      __syncthreads();
      fl.flush(g0, m);
    }
  }

  if (active) {
    // After n draws the ring phase is m: canonical V[k] = R[(k + m) % 97].
#pragma unroll
    for (int r = 0; r < 97; r++) {
      const int k = (r - m + 97) % 97;
      d.state[(uint64_t)k * nr + row] = R[r] & 0xFFFFFFu;
    }
    d.state[97 * nr + row] = C;
  }
}

template <int T, bool F32>
__global__ void __launch_bounds__(T, 512 / T) k_fill_ranmar(const FillDesc d) {
  extern __shared__ uint32_t smem[];
  ranmar_rows<T, F32, false>(d, (uint64_t)blockIdx.x * T, smem);
}

// Batched RANMAR fills: one block per item (T streams of one request),
// items ordered longest first.  With the 97-word lag table in registers a
// persistent loop around the body does not fit the register budget, so
// here the hardware block scheduler hands out the items in order.
template <int T, bool F32>
__global__ void __launch_bounds__(T, 512 / T) k_batch_ranmar(const BatchQueue q) {
  extern __shared__ uint32_t smem[];
  const BatchItem si = q.items[blockIdx.x];
  ranmar_rows<T, F32, true>(q.reqs[si.req].d, si.row0, smem);
}

template <int T, bool F32>
static cudaError_t launch_bm(const BatchQueue& q, cudaStream_t s) {
  constexpr size_t bytes = (size_t)97 * (T + 1) * sizeof(uint32_t);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_batch_ranmar<T, F32>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  k_batch_ranmar<T, F32><<<q.n_items, T, bytes, s>>>(q);
  return cudaGetLastError();
}

cudaError_t launch_batch_ranmar(const BatchQueue& q, Tile t, bool f32, cudaStream_t s) {
  if (q.n_items == 0) return cudaSuccess;
  if (t.threads == 128) return f32 ? launch_bm<128, true>(q, s) : launch_bm<128, false>(q, s);
  return f32 ? launch_bm<64, true>(q, s) : launch_bm<64, false>(q, s);
}

template <int T, bool F32>
static cudaError_t launch_m(const FillDesc& d, cudaStream_t s) {
  constexpr size_t bytes = (size_t)97 * (T + 1) * sizeof(uint32_t);
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
