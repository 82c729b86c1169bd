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
#include "batch.cuh"

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

template <class G, int OM>
__device__ __forceinline__ uint32_t lj_conv(uint32_t v) {
  if constexpr (OM == OUT_F32) return as_f32_bits<G::SH>(v);
  else return v;   // u32, or a raw draw paired at the store
}

// Per-warp constants of one call: multipliers to a lane's first draw, to
// the next 128-draw block and over the whole call (n draws).
template <class G>
struct LjConst {
  uint32_t lane_mul[G::NC], block_mul[G::NC], fin_mul[G::NC];
  __device__ __forceinline__ void init(int lane, uint64_t n) {
#pragma unroll
    for (int c = 0; c < G::NC; c++) {
      lane_mul[c] = G::pow(c, 4 * lane + 1);
      block_mul[c] = G::pow(c, 128);
      fin_mul[c] = G::pow(c, n);
    }
  }
};

// One row (stream, or jump chunk whose start components are `base`) by one
// warp: draws 0 .. nv-1 written to orow (row start), 16-byte stores when vec.
template <class G, int OM>
__device__ __forceinline__ void lj_row(const LjConst<G>& K, const uint32_t (&base)[G::NC], int lane,
                                       uint32_t* orow, uint64_t nv, bool vec, const FillDesc& d,
                                       uint64_t erow) {
  constexpr int NC = G::NC;
  uint32_t s[NC];
#pragma unroll
  for (int c = 0; c < NC; c++) s[c] = G::mul(c, K.lane_mul[c], base[c]);
  orow += 4 * lane;
  erow += 4 * lane;
  for (uint64_t c0 = 0; c0 < nv; c0 += 128) {
    uint32_t t[NC], o[4];
#pragma unroll
    for (int c = 0; c < NC; c++) t[c] = s[c];
    o[0] = lj_conv<G, OM>(G::out(t));
#pragma unroll
    for (int i = 1; i < 4; i++) {
#pragma unroll
      for (int c = 0; c < NC; c++) t[c] = G::step(c, t[c]);
      o[i] = lj_conv<G, OM>(G::out(t));
    }
    if constexpr (OM == OUT_ISING) {
      if (c0 + 128 <= nv) {
        put4<OM, 31>(d, nullptr, erow + c0, make_uint4(o[0], o[1], o[2], o[3]));
      } else {
#pragma unroll
        for (int i = 0; i < 4; i++)
          if (c0 + 4 * lane + i < nv) put1<OM>(d, nullptr, erow + c0 + i, o[i]);
      }
    } else if (vec && c0 + 128 <= nv) {
      st_chunk<OM, 31>(orow + c0, make_uint4(o[0], o[1], o[2], o[3]));
    } else if constexpr (OM == OUT_F64) {   // nv is even: pairs are whole
#pragma unroll
      for (int i = 0; i < 4; i += 2)
        if (c0 + 4 * lane + i < nv) st_pair<31>(orow + c0 + i, o[i], o[i + 1]);
    } else {
#pragma unroll
      for (int i = 0; i < 4; i++)
        if (c0 + 4 * lane + i < nv) st_out(orow + c0 + i, o[i]);
    }
#pragma unroll
    for (int c = 0; c < NC; c++) s[c] = G::mul(c, s[c], K.block_mul[c]);
  }
}

// Stream `row` of a handle fill: load its state, write its row, store the
// state advanced by n draws (lane 0).
template <class G, int OM>
__device__ __forceinline__ void lj_stream(const LjConst<G>& K, const FillDesc& d, uint64_t row, int lane) {
  constexpr int NC = G::NC;
  uint32_t base[NC];
#pragma unroll
  for (int c = 0; c < NC; c++) base[c] = d.state[c * d.n_rows + row];
  uint64_t nv = d.n_per;
  if (d.limit - row * d.pitch < nv) nv = d.limit - row * d.pitch;
  uint32_t* out = static_cast<uint32_t*>(d.out);
  const bool vec = ((d.pitch & 3) == 0) && ((reinterpret_cast<uintptr_t>(out) & 15) == 0);
  lj_row<G, OM>(K, base, lane, out + row * d.pitch, nv, vec, d, row * d.pitch);
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < NC; c++) d.state[c * d.n_rows + row] = G::mul(c, base[c], K.fin_mul[c]);
  }
}

template <class G, int WPB, int OM>
__global__ void __launch_bounds__(WPB * 32) k_fill_lj(const FillDesc d) {
  constexpr int NC = G::NC;
  const int lane = threadIdx.x & 31;
  const uint64_t nwarps = (uint64_t)gridDim.x * WPB;
  const uint64_t wrow = (uint64_t)blockIdx.x * WPB + (threadIdx.x >> 5);
  LjConst<G> K;
  K.init(lane, d.n_per);
  if (!d.jump) {
    for (uint64_t row = wrow; row < d.n_rows; row += nwarps) lj_stream<G, OM>(K, d, row, lane);
    return;
  }
  // Jump fill: chunk r starts at a^(r L) x0; this warp's chunks are nwarps apart.
  uint32_t jrow[NC], jstep[NC];
#pragma unroll
  for (int c = 0; c < NC; c++) {
    jrow[c] = G::mul(c, G::pow(c, wrow * d.pitch), G::x0_part(c, d.x0));
    jstep[c] = G::pow(c, nwarps * d.pitch);
  }
  uint32_t* out = static_cast<uint32_t*>(d.out);
  const bool vec_ok = ((d.pitch & 3) == 0) && ((reinterpret_cast<uintptr_t>(out) & 15) == 0);
  for (uint64_t row = wrow; row < d.n_rows; row += nwarps) {
    uint64_t nv = d.n_per;
    if (d.limit - row * d.pitch < nv) nv = d.limit - row * d.pitch;
    lj_row<G, OM>(K, jrow, lane, out + row * d.pitch, nv, vec_ok && ((row * d.pitch) & 3) == 0, d,
                  row * d.pitch);
#pragma unroll
    for (int c = 0; c < NC; c++) jrow[c] = G::mul(c, jrow[c], jstep[c]);
  }
}

// Batched fills of GGL and RANECU handles: a warp pops an item (up to 8
// streams of one request) and fills its streams one after the other.
template <int WPB>
__global__ void __launch_bounds__(WPB * 32) k_batch_mlcg(const BatchQueue q) {
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  __shared__ FillDesc desc[WPB];
  for (;;) {
    const uint32_t it = pop_warp(q.counter);
    if (it >= q.n_items) break;
    const BatchItem I = q.items[it];
    const BatchReq& r = q.reqs[I.req];
    FillDesc& d = desc[wi];
    __syncwarp();
    load_desc(&d, r.d, lane, 32);
    __syncwarp();
    if (r.gen == GGL) {
      LjConst<GglLJ> K;
      K.init(lane, d.n_per);
      for (uint32_t k = 0; k < I.rows; k++) {
        if (d.mode == OUT_F32) lj_stream<GglLJ, OUT_F32>(K, d, I.row0 + k, lane);
        else lj_stream<GglLJ, OUT_U32>(K, d, I.row0 + k, lane);
      }
    } else {
      LjConst<RanecuLJ> K;
      K.init(lane, d.n_per);
      for (uint32_t k = 0; k < I.rows; k++) {
        if (d.mode == OUT_F32) lj_stream<RanecuLJ, OUT_F32>(K, d, I.row0 + k, lane);
        else lj_stream<RanecuLJ, OUT_U32>(K, d, I.row0 + k, lane);
      }
    }
  }
}

cudaError_t launch_batch_mlcg(const BatchQueue& q, Tile t, cudaStream_t s) {
  (void)t;
  if (q.n_items == 0) return cudaSuccess;
  const uint32_t cap = (uint32_t)sm_count() * (2048 / 128);
  const uint32_t need = (q.n_items + 3) / 4;
  k_batch_mlcg<4><<<need < cap ? need : cap, 128, 0, s>>>(q);
  return cudaGetLastError();
}

template <class G, int WPB, int OM>
static cudaError_t launch_lj(const FillDesc& d, cudaStream_t s) {
  const uint64_t need = (d.n_rows + WPB - 1) / WPB;
  const uint64_t resident = (uint64_t)sm_count() * (2048 / (WPB * 32));
  const unsigned grid = (unsigned)(need < resident ? need : resident);
  k_fill_lj<G, WPB, OM><<<grid, WPB * 32, 0, s>>>(d);
  return cudaGetLastError();
}

template <class G>
static cudaError_t launch_lj_g(const FillDesc& d, Tile t, cudaStream_t s) {
  return with_mode(d.mode, [&](auto m) {
    return t.threads == 256 ? launch_lj<G, 8, decltype(m)::value>(d, s)
                            : launch_lj<G, 4, decltype(m)::value>(d, s);
  });
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
