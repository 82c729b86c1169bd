// k_mlcg.cu -- bulk and jump-ahead fills of the two multiplicative
// congruential generators, GGL (Section 3.2) and RANECU (Section 3.4).
//
// These two generators jump ahead cheaply: x_{n+k} = a^k x_n mod m
// (Appendix A, eq. MLCG), for RANECU per component.  So one warp owns one
// stream (or one chunk of a jump fill) at a time and its 32 lanes cover 128
// consecutive draws: lane l holds draws 4l .. 4l+3 of the current 128-draw
// block -- the first from the block's start times the per-lane constant
// a^(4l+1), the other three by single steps -- and the next block starts
// a^128 further on.  Every warp store is then one 512-byte run of the
// stream's output row, with no shared-memory staging and no barriers.
// Rows are taken in a grid-stride loop.  Since every stream of a call
// advances by the same n, the state left after the call is the stored state
// times a^n, one multiplication per row with a^n computed once per warp.
#include "common.cuh"

namespace prng {

// GGL: one component, x <- 16807 x mod (2^31 - 1).
struct GglLJ {
  static constexpr int NC = 1, SH = 7;
  static __device__ __forceinline__ uint32_t step(int, uint32_t x) { return mlcg_step<16807u, 1u>(x); }
  static __device__ __forceinline__ uint32_t mul(int, uint32_t x, uint32_t y) { return mulmod_pm<1u>(x, y); }
  static __device__ __forceinline__ uint32_t pow(int, uint64_t e) { return powmod_pm<1u>(16807u, e); }
  static __device__ __forceinline__ uint32_t x0_part(int, uint64_t x0) { return (uint32_t)x0; }
  static __device__ __forceinline__ uint32_t out(const uint32_t (&s)[NC]) { return s[0]; }
};

// RANECU: components 40014 mod 2147483563 and 40692 mod 2147483399,
// combined as s1 - s2, plus m1 - 1 when not positive.
struct RanecuLJ {
  static constexpr int NC = 2, SH = 7;
  static __device__ __forceinline__ uint32_t step(int c, uint32_t x) {
    return c == 0 ? mlcg_step<40014u, 85u>(x) : mlcg_step<40692u, 249u>(x);
  }
  static __device__ __forceinline__ uint32_t mul(int c, uint32_t x, uint32_t y) {
    return c == 0 ? mulmod_pm<85u>(x, y) : mulmod_pm<249u>(x, y);
  }
  static __device__ __forceinline__ uint32_t pow(int c, uint64_t e) {
    return c == 0 ? powmod_pm<85u>(40014u, e) : powmod_pm<249u>(40692u, e);
  }
  static __device__ __forceinline__ uint32_t x0_part(int c, uint64_t x0) {
    return c == 0 ? (uint32_t)(x0 & 0xFFFFFFFFu) : (uint32_t)(x0 >> 32);
  }
  static __device__ __forceinline__ uint32_t out(const uint32_t (&s)[NC]) {
    int32_t z = (int32_t)s[0] - (int32_t)s[1];
    z += (z < 1) ? 2147483562 : 0;
    return (uint32_t)z;
  }
};

template <class G, bool F32>
__device__ __forceinline__ uint32_t lj_conv(uint32_t v) {
  if constexpr (F32) return as_f32_bits<G::SH>(v);
  else return v;
}

template <class G, int WPB, bool F32>
__global__ void __launch_bounds__(WPB * 32) k_fill_lj(const FillDesc d) {
  constexpr int NC = G::NC;
  const int lane = threadIdx.x & 31;
  const uint64_t nwarps = (uint64_t)gridDim.x * WPB;
  const uint64_t wrow = (uint64_t)blockIdx.x * WPB + (threadIdx.x >> 5);
  const uint64_t n = d.n_per;
  uint32_t* out = static_cast<uint32_t*>(d.out);
  const bool vec_ok = ((d.pitch & 3) == 0) && ((reinterpret_cast<uintptr_t>(out) & 15) == 0);

  uint32_t lane_mul[NC], block_mul[NC], fin_mul[NC], jrow[NC], jstep[NC];
#pragma unroll
  for (int c = 0; c < NC; c++) {
    lane_mul[c] = G::pow(c, 4 * lane + 1);
    block_mul[c] = G::pow(c, 128);
    fin_mul[c] = G::pow(c, n);
    if (d.jump) {  // chunk r starts at a^(r L) x0; this warp's rows are nwarps apart
      jrow[c] = G::mul(c, G::pow(c, wrow * d.pitch), G::x0_part(c, d.x0));
      jstep[c] = G::pow(c, nwarps * d.pitch);
    } else {
      jrow[c] = jstep[c] = 0;
    }
  }

  for (uint64_t row = wrow; row < d.n_rows; row += nwarps) {
    uint32_t base[NC], s[NC];
#pragma unroll
    for (int c = 0; c < NC; c++) {
      base[c] = d.jump ? jrow[c] : d.state[c * d.n_rows + row];
      s[c] = G::mul(c, lane_mul[c], base[c]);
    }
    uint64_t nv = n;  // draws of this row to write (a jump fill's last chunk is shorter)
    if (d.limit - row * d.pitch < nv) nv = d.limit - row * d.pitch;
    uint32_t* orow = out + row * d.pitch + 4 * lane;
    const bool vec = vec_ok && ((row * d.pitch) & 3) == 0;
    for (uint64_t c0 = 0; c0 < nv; c0 += 128) {
      uint32_t t[NC], o[4];
#pragma unroll
      for (int c = 0; c < NC; c++) t[c] = s[c];
      o[0] = lj_conv<G, F32>(G::out(t));
#pragma unroll
      for (int i = 1; i < 4; i++) {
#pragma unroll
        for (int c = 0; c < NC; c++) t[c] = G::step(c, t[c]);
        o[i] = lj_conv<G, F32>(G::out(t));
      }
      if (vec && c0 + 128 <= nv) {
        st_out4(orow + c0, make_uint4(o[0], o[1], o[2], o[3]));
      } else {
#pragma unroll
        for (int i = 0; i < 4; i++)
          if (c0 + 4 * lane + i < nv) st_out(orow + c0 + i, o[i]);
      }
#pragma unroll
      for (int c = 0; c < NC; c++) s[c] = G::mul(c, s[c], block_mul[c]);
    }
    if (!d.jump && lane == 0) {
#pragma unroll
      for (int c = 0; c < NC; c++) d.state[c * d.n_rows + row] = G::mul(c, base[c], fin_mul[c]);
    }
    if (d.jump) {
#pragma unroll
      for (int c = 0; c < NC; c++) jrow[c] = G::mul(c, jrow[c], jstep[c]);
    }
  }
}

static int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 1;
  }
  return n;
}

template <class G, int WPB, bool F32>
static cudaError_t launch_lj(const FillDesc& d, cudaStream_t s) {
  const uint64_t need = (d.n_rows + WPB - 1) / WPB;
  const uint64_t resident = (uint64_t)sm_count() * (2048 / (WPB * 32));
  const unsigned grid = (unsigned)(need < resident ? need : resident);
  k_fill_lj<G, WPB, F32><<<grid, WPB * 32, 0, s>>>(d);
  return cudaGetLastError();
}

template <class G>
static cudaError_t launch_lj_g(const FillDesc& d, Tile t, cudaStream_t s) {
  if (t.threads == 256) return d.f32 ? launch_lj<G, 8, true>(d, s) : launch_lj<G, 8, false>(d, s);
  return d.f32 ? launch_lj<G, 4, true>(d, s) : launch_lj<G, 4, false>(d, s);
}

cudaError_t launch_fill_mlcg(int gen, const FillDesc& d, Tile t, cudaStream_t s) {
  if (d.n_rows == 0 || d.n_per == 0) return cudaSuccess;
  if (gen == GGL) return launch_lj_g<GglLJ>(d, t, s);
  if (gen == RANECU) return launch_lj_g<RanecuLJ>(d, t, s);
  return cudaErrorInvalidValue;
}

// Skip of the MLCG generators in closed form: x <- a^k x mod m.
__global__ void k_skip_mlcg(int gen, uint32_t* state, uint64_t n, uint64_t k) {
  const uint64_t row = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  if (gen == GGL) {
    state[row] = mulmod_pm<1>(powmod_pm<1>(16807u, k), state[row]);
  } else {
    state[row] = mulmod_pm<85u>(powmod_pm<85u>(40014u, k), state[row]);
    state[n + row] = mulmod_pm<249u>(powmod_pm<249u>(40692u, k), state[n + row]);
  }
}

cudaError_t launch_skip_mlcg(int gen, uint32_t* state, uint64_t n, uint64_t k, cudaStream_t s) {
  if (n == 0 || k == 0) return cudaSuccess;
  k_skip_mlcg<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(gen, state, n, k);
  return cudaGetLastError();
}

}  // namespace prng
