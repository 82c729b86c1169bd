// k_mt.cu -- MT19937 fill and skip (Section 3.7; Appendix A, "Mersenne
// twister").
//
// One warp per stream, its 624-word table in shared memory.  The twist
// X_{n+624} = X_{n+397} ^ (X_n^upper | X_{n+1}^lower) A is done in place in
// 20 warp-wide chunks of 32 consecutive entries, in increasing order: entry
// k reads old k and k+1 and either old k+397 (k < 227) or new k-227
// (k >= 227, produced at least one chunk earlier), so a chunk needs only a
// __syncwarp between its reads and its writes.  Each new word is tempered
// and stored by the lane that produced it, so the 32 lanes write 32
// consecutive outputs of the stream's row: coalesced without staging.
#include "common.cuh"

namespace prng {

__device__ __forceinline__ uint32_t mt_temper(uint32_t t) {
  t ^= t >> 11;
  t ^= (t << 7) & 0x9D2C5680u;
  t ^= (t << 15) & 0xEFC60000u;
  t ^= t >> 18;
  return t;
}

template <bool F32>
__device__ __forceinline__ uint32_t mt_conv(uint32_t t) {
  if constexpr (F32) return as_f32_bits<8>(t);
  else return t;
}

template <int WPB, bool F32>
__global__ void __launch_bounds__(WPB * 32) k_fill_mt(const FillDesc d) {
  __shared__ uint32_t table[WPB][624];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const uint64_t row = (uint64_t)blockIdx.x * WPB + wi;
  if (row >= d.n_rows) return;  // whole warp leaves; no CTA-wide barriers below
  uint32_t* s = table[wi];
  uint32_t* gs = d.state + row * 624;
  for (int k = lane; k < 624; k += 32) s[k] = gs[k];
  __syncwarp();

  uint32_t* out = static_cast<uint32_t*>(d.out);
  const bool store = out != nullptr;
  uint32_t* orow = store ? out + row * d.pitch : nullptr;
  const uint64_t n = d.n_per;
  uint64_t j = 0;
  const uint32_t mti = d.pos;
  if (mti < 624 && n > 0) {  // rest of the current table
    const uint64_t h = (624 - mti) < n ? (624 - mti) : n;
    if (store)
      for (uint64_t k = lane; k < h; k += 32) st_out(orow + k, mt_conv<F32>(mt_temper(s[mti + k])));
    j = h;
  }
  while (j < n) {
    const uint64_t take = (n - j) < 624 ? (n - j) : 624;
#pragma unroll 4
    for (int k0 = 0; k0 < 640; k0 += 32) {
      const int k = k0 + lane;
      uint32_t a = 0, b = 0, f = 0;
      if (k < 624) {
        a = s[k];
        b = s[k == 623 ? 0 : k + 1];
        f = s[k < 227 ? k + 397 : k - 227];
      }
      __syncwarp();
      if (k < 624) {
        const uint32_t y = (a & 0x80000000u) | (b & 0x7FFFFFFFu);
        const uint32_t v = f ^ (y >> 1) ^ ((y & 1u) ? 0x9908B0DFu : 0u);
        s[k] = v;
        if (store && (uint64_t)k < take) st_out(orow + j + k, mt_conv<F32>(mt_temper(v)));
      }
      __syncwarp();
    }
    j += take;
  }
  for (int k = lane; k < 624; k += 32) gs[k] = s[k];
}

template <int WPB, bool F32>
static cudaError_t launch_mt(const FillDesc& d, cudaStream_t s) {
  const uint64_t grid = (d.n_rows + WPB - 1) / WPB;
  k_fill_mt<WPB, F32><<<(unsigned)grid, WPB * 32, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_fill_mt(const FillDesc& d, Tile t, cudaStream_t s) {
  if (d.n_rows == 0 || d.n_per == 0) return cudaSuccess;
  if (t.threads == 64) return d.f32 ? launch_mt<2, true>(d, s) : launch_mt<2, false>(d, s);
  if (t.threads == 256) return d.f32 ? launch_mt<8, true>(d, s) : launch_mt<8, false>(d, s);
  return d.f32 ? launch_mt<4, true>(d, s) : launch_mt<4, false>(d, s);
}

}  // namespace prng
