// k_ranmar.cu -- RANMAR fill and skip (Section 3.5; Appendix A, "RANMAR").
//
// One warp per stream.  The two table indices (i97, j97) fall together by
// one per draw and are the same for every stream, so the state is kept in
// canonical order (V[0] = the entry overwritten next, V[k] = x_{n-97+k}
// before draw n) and the lagged part is x_n = x_{n-97} - x_{n-33} mod 2^24.
// Both lags exceed a warp's width, so a warp computes 32 consecutive draws
// per step, one per lane, from a 128-slot ring of the stream's recent lag
// values in shared memory, and writes them as one coalesced 128-byte run of
// the stream's output row.  The Weyl term C_n = C_{n-1} - D mod M is
// evaluated per draw as an offset of the step group's entry value by a
// per-lane constant, so no draw waits on the previous one.
#include "batch.cuh"

namespace prng {

constexpr uint32_t kRanmarD = 7654321u;    // Section 3.5: RM_CD * 2^24
constexpr uint32_t kRanmarM = 16777213u;   // Section 3.5: RM_CM * 2^24

// C0 after `steps` more draws.
__device__ __forceinline__ uint32_t ranmar_advance_c(uint32_t C0, uint32_t steps) {
  const uint32_t kd = (uint32_t)(((uint64_t)steps * kRanmarD) % kRanmarM);
  const int32_t c = (int32_t)C0 - (int32_t)kd;
  return c < 0 ? (uint32_t)(c + (int32_t)kRanmarM) : (uint32_t)c;
}

template <int OM>
__device__ __forceinline__ uint32_t rm_conv(uint32_t x) {
  if constexpr (OM == OUT_F32) return __float_as_uint(__uint2float_rn(x) * 0x1p-24f);
  else return x;
}

// Ring slots per stream: 128 for the lag table, slot 128 for C, padding to
// 132 words so that the cooperative state load (eight streams side by side)
// hits 32 different banks.
constexpr int kRanmarRing = 132;

// One pass over `rows` <= NW streams [row0, row0 + rows), one warp each.
//
// The lags (97, 33) both exceed 32, so the 32 draws x_n .. x_{n+31} depend
// only on earlier draws: lane l computes x_{n+l}, and a warp advances its
// stream 32 draws per step.  The stream's last 128 lag values sit in a
// shared ring, x_m in slot (m + 97) mod 128, so the canonical table V[k] =
// x_{k-97} loads to slots 0..96 unchanged; step draws x_n read slots n mod
// 128 (lag 97) and (n + 64) mod 128 (lag 33) and write slot (n + 97) mod 128.
// Every output store is one 128-byte run of the stream's row, with no
// staging.  The state moves between HBM and the rings through one
// cooperative pass of the block (eight consecutive streams per 32-byte
// sector).
template <int NW, int OM, bool LIMITED>
__device__ __forceinline__ void ranmar_warps(const FillDesc& d, uint64_t row0, int rows,
                                             uint32_t* smem) {
  constexpr int RS = kRanmarRing;
  const uint64_t nr = d.n_rows;
  for (int e = threadIdx.x; e < 98 * NW; e += NW * 32) {
    const int j = e / NW, w = e % NW;
    if (w < rows) smem[w * RS + (j < 97 ? j : 128)] = d.state[(uint64_t)j * nr + row0 + w];
  }
  __syncthreads();

  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const uint64_t n = d.n_per;
  if (w < rows) {
    uint32_t* ring = smem + w * RS;
    uint32_t C = ring[128];
    uint32_t* out = static_cast<uint32_t*>(d.out);
    const bool store = out != nullptr;
    const uint64_t rbase = (row0 + w) * d.pitch;   // element index of the row's first draw
    uint32_t* orow = store ? out + rbase : nullptr;
    uint32_t kd[4];                                // ((32 s + l + 1) D) mod M
    uint32_t* wp[4];                               // slot of this lane's draw in step s
#pragma unroll
    for (int s = 0; s < 4; s++) {
      kd[s] = (uint32_t)(((uint64_t)(32 * s + l + 1) * kRanmarD) % kRanmarM);
      wp[s] = ring + ((32 * s + 97 + l) & 127);
    }
    const uint32_t* rl = ring + l;
    // Lane l's draw of step s: Y = x_{n-97} - x_{n-33}, kept modulo 2^32
    // (only its low 24 bits matter).  The Weyl term after it is C = C_group
    // - kd[s] mod M: with c = C_group - kd[s] as a 32-bit word, C = c when no
    // wrap happened and c + M otherwise; since M = 2^24 - 3 and c >> 30 is 3
    // exactly when it wrapped, X = (Y - C) mod 2^24 = (Y - c + (c >> 30))
    // mod 2^24.
    auto out_word = [&](uint32_t y, int s) {
      const uint32_t c = C - kd[s];
      return rm_conv<OM>((y - c + (c >> 30)) & 0xFFFFFFu);
    };
    // Store of the step's 32 words (lanes with `on`); doubles pair lane l
    // (even) with lane l + 1 (n is even, so a pair is never cut).
    auto emit = [&](uint64_t col0, uint32_t v, bool on) {
      const uint64_t col = col0 + l;
      if constexpr (OM == OUT_F64) {
        const uint32_t vb = __shfl_down_sync(0xFFFFFFFFu, v, 1);
        if (on && !(l & 1) && (!LIMITED || rbase + col < d.limit)) st_pair<24>(orow + col, v, vb);
      } else {
        if (on && (!LIMITED || rbase + col < d.limit)) put1<OM>(d, orow + col, rbase + col, v);
      }
    };
    // Doubles of a 64-draw pair of steps, one per lane: lane l takes draws
    // 2l and 2l + 1 of the pair (of the first step for l < 16, of the second
    // for l >= 16), so every lane assembles a double and the warp writes 256
    // contiguous bytes.
    auto emit_pairs = [&](uint64_t col0, uint32_t va, uint32_t vb) {
      const int src = (2 * l) & 31;
      const uint32_t a0 = __shfl_sync(0xFFFFFFFFu, va, src);
      const uint32_t b0 = __shfl_sync(0xFFFFFFFFu, va, src + 1);
      const uint32_t a1 = __shfl_sync(0xFFFFFFFFu, vb, src);
      const uint32_t b1 = __shfl_sync(0xFFFFFFFFu, vb, src + 1);
      st_pair<24>(orow + col0 + 2 * l, l < 16 ? a0 : a1, l < 16 ? b0 : b1);
    };
    uint64_t g = 0;
    for (; g + 128 <= n; g += 128) {
      uint32_t v[4];
#pragma unroll
      for (int s = 0; s < 4; s++) {
        const uint32_t y = rl[32 * s] - rl[32 * ((s + 2) & 3)];
        *wp[s] = y;
        __syncwarp();
        v[s] = out_word(y, s);
        if constexpr (OM != OUT_F64 || LIMITED)
          if (store) emit(g + 32 * s, v[s], true);
      }
      if constexpr (OM == OUT_F64 && !LIMITED) {
        if (store) {
          emit_pairs(g, v[0], v[1]);
          emit_pairs(g + 64, v[2], v[3]);
        }
      }
      C = ranmar_advance_c(C, 128);
    }
    const int rem = (int)(n - g);
    if (rem > 0) {
#pragma unroll
      for (int s = 0; s < 4; s++) {
        if (32 * s < rem) {
          const bool on = 32 * s + l < rem;
          uint32_t y = 0;
          if (on) {
            y = rl[32 * s] - rl[32 * ((s + 2) & 3)];
            *wp[s] = y;
          }
          __syncwarp();
          if (store) emit(g + 32 * s, on ? out_word(y, s) : 0u, on);
        }
      }
      C = ranmar_advance_c(C, (uint32_t)rem);
    }
    __syncwarp();
    if (l == 0) ring[128] = C;
  }
  __syncthreads();

  // Canonical order after n draws: V[k] = x_{n-97+k}, in slot (n + k) mod 128.
  const int off = (int)(n & 127);
  for (int e = threadIdx.x; e < 98 * NW; e += NW * 32) {
    const int j = e / NW, w2 = e % NW;
    if (w2 < rows) {
      const uint32_t v = j < 97 ? smem[w2 * RS + ((off + j) & 127)] & 0xFFFFFFu : smem[w2 * RS + 128];
      d.state[(uint64_t)j * nr + row0 + w2] = v;
    }
  }
}

template <int T, int OM>
__global__ void __launch_bounds__(T) k_fill_ranmar(const FillDesc d) {
  __shared__ uint32_t smem[(T / 32) * kRanmarRing];
  const uint64_t row0 = (uint64_t)blockIdx.x * (T / 32);
  const uint64_t left = d.n_rows - row0;
  ranmar_warps<T / 32, OM, false>(d, row0, left < (uint64_t)(T / 32) ? (int)left : T / 32, smem);
}

// Batched RANMAR fills: one block per item (up to T / 32 streams of one
// request, items ordered longest first, handed out in order by the block
// scheduler).
template <int T, bool F32>
__global__ void __launch_bounds__(T) k_batch_ranmar(const BatchQueue q) {
  __shared__ uint32_t smem[(T / 32) * kRanmarRing];
  const BatchItem si = q.items[blockIdx.x];
  __shared__ FillDesc sd;
  load_desc(&sd, q.reqs[si.req].d, threadIdx.x, T);
  __syncthreads();
  ranmar_warps<T / 32, F32 ? OUT_F32 : OUT_U32, true>(sd, si.row0, (int)si.rows, smem);
}

template <int T, bool F32>
static cudaError_t launch_bm(const BatchQueue& q, cudaStream_t s) {
  k_batch_ranmar<T, F32><<<q.n_items, T, 0, s>>>(q);
  return cudaGetLastError();
}

cudaError_t launch_batch_ranmar(const BatchQueue& q, Tile t, bool f32, cudaStream_t s) {
  if (q.n_items == 0) return cudaSuccess;
  if (t.threads == 128) return f32 ? launch_bm<128, true>(q, s) : launch_bm<128, false>(q, s);
  return f32 ? launch_bm<256, true>(q, s) : launch_bm<256, false>(q, s);
}

template <int T, int OM>
static cudaError_t launch_m(const FillDesc& d, cudaStream_t s) {
  const uint64_t grid = (d.n_rows + T / 32 - 1) / (T / 32);
  if (grid > 0x7FFFFFFFull) return cudaErrorInvalidValue;
  k_fill_ranmar<T, OM><<<(unsigned)grid, T, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_fill_ranmar(const FillDesc& d, Tile t, cudaStream_t s) {
  if (d.n_rows == 0 || d.n_per == 0) return cudaSuccess;
  return with_mode(d.mode, [&](auto m) {
    return t.threads == 128 ? launch_m<128, decltype(m)::value>(d, s)
                            : launch_m<256, decltype(m)::value>(d, s);
  });
}

}  // namespace prng
