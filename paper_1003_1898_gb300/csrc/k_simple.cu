// k_simple.cu -- bulk fill for the register-state generators GGL (Section 3.2),
// XOR128 (Section 3.3) and RANECU (Section 3.4), their jump-ahead
// single-sequence fill, and the O(log k) skip of the two MLCG generators.
//
// One thread owns one stream (or one jump chunk) with its state in
// registers.  Output is stream-major, so a warp's 32 streams write 32
// different rows: each thread drafts K consecutive draws into its row of a
// shared-memory tile with 16-byte stores, then the CTA writes the tile out
// row by row (a warp covers 4 rows x 128 contiguous bytes per 16-byte store),
// which turns the per-thread sequences into coalesced HBM writes.  The tile
// is double-buffered so one barrier per tile suffices.
#include "common.cuh"

namespace prng {

struct GglGen {
  static constexpr int SH = 7;
  uint32_t x;
  __device__ __forceinline__ void load(const uint32_t* st, uint64_t n, uint64_t row) { x = st[row]; }
  __device__ __forceinline__ void store(uint32_t* st, uint64_t n, uint64_t row) const { st[row] = x; }
  // Chunk start x0 a^e mod m (Appendix A, eq. MLCG in closed form).
  __device__ __forceinline__ void jump_init(uint64_t x0, uint64_t e) {
    x = mulmod_pm<1>(powmod_pm<1>(16807u, e), (uint32_t)x0);
  }
  __device__ __forceinline__ void zero() { x = 1; }
  // x <- 16807 x mod (2^31 - 1)  (Section 3.2 constants).
  __device__ __forceinline__ uint32_t next() {
    x = mlcg_step<16807u, 1u>(x);
    return x;
  }
};

struct Xor128Gen {
  static constexpr int SH = 8;
  uint32_t x, y, z, w;
  __device__ __forceinline__ void load(const uint32_t* st, uint64_t n, uint64_t row) {
    x = st[row];
    y = st[n + row];
    z = st[2 * n + row];
    w = st[3 * n + row];
  }
  __device__ __forceinline__ void store(uint32_t* st, uint64_t n, uint64_t row) const {
    st[row] = x;
    st[n + row] = y;
    st[2 * n + row] = z;
    st[3 * n + row] = w;
  }
  __device__ __forceinline__ void jump_init(uint64_t, uint64_t) {}
  __device__ __forceinline__ void zero() { x = y = z = 0; w = 1; }
  // Appendix A, "XORShift", scalar form of XOR128 with shifts 11, 19, 8.
  __device__ __forceinline__ uint32_t next() {
    const uint32_t t = x ^ (x << 11);
    x = y;
    y = z;
    z = w;
    w = (w ^ (w >> 19)) ^ (t ^ (t >> 8));
    return w;
  }
};

struct RanecuGen {
  static constexpr int SH = 7;
  uint32_t s1, s2;
  __device__ __forceinline__ void load(const uint32_t* st, uint64_t n, uint64_t row) {
    s1 = st[row];
    s2 = st[n + row];
  }
  __device__ __forceinline__ void store(uint32_t* st, uint64_t n, uint64_t row) const {
    st[row] = s1;
    st[n + row] = s2;
  }
  // Each component jumped separately: s_j a_j^e mod m_j.
  __device__ __forceinline__ void jump_init(uint64_t x0, uint64_t e) {
    s1 = mulmod_pm<85u>(powmod_pm<85u>(40014u, e), (uint32_t)(x0 & 0xFFFFFFFFu));
    s2 = mulmod_pm<249u>(powmod_pm<249u>(40692u, e), (uint32_t)(x0 >> 32));
  }
  __device__ __forceinline__ void zero() { s1 = s2 = 1; }
  // Section 3.4: m1 = 2147483563 = 2^31 - 85, m2 = 2147483399 = 2^31 - 249;
  // combination z = s1 - s2, plus m1 - 1 when z < 1 (Appendix A, "Multiple
  // recursive generators").
  __device__ __forceinline__ uint32_t next() {
    s1 = mlcg_step<40014u, 85u>(s1);
    s2 = mlcg_step<40692u, 249u>(s2);
    int32_t z = (int32_t)s1 - (int32_t)s2;
    z += (z < 1) ? 2147483562 : 0;
    return (uint32_t)z;
  }
};

template <class G, bool F32>
__device__ __forceinline__ uint32_t conv(uint32_t v) {
  if constexpr (F32) return as_f32_bits<G::SH>(v);
  else return v;
}

template <class G, int T, int K, bool F32>
__global__ void __launch_bounds__(T) k_fill_simple(const FillDesc d) {
  constexpr int SP = K + 4;  // row pitch in words: 16-byte stores of 8 rows hit 8 distinct bank quads
  extern __shared__ __align__(16) uint32_t smem[];  // two tiles of T * SP words
  const int tid = threadIdx.x;
  const uint64_t row0 = (uint64_t)blockIdx.x * T;
  const uint64_t row = row0 + tid;
  const bool active = row < d.n_rows;

  G g;
  if (!active) g.zero();
  else if (d.jump) g.jump_init(d.x0, row * d.pitch);
  else g.load(d.state, d.n_rows, row);

  uint32_t* out = static_cast<uint32_t*>(d.out);
  const bool vec_ok = ((d.pitch & 3) == 0) && ((reinterpret_cast<uintptr_t>(out) & 15) == 0);
  const uint64_t last_row = (row0 + T < d.n_rows ? row0 + T : d.n_rows) - 1;
  const uint64_t n = d.n_per;
  int buf = 0;
  for (uint64_t c0 = 0; c0 < n; c0 += K) {
    const int w = (n - c0 < (uint64_t)K) ? (int)(n - c0) : K;
    uint32_t* const t = smem + buf * (T * SP);
    uint32_t* my = t + tid * SP;
    if (w == K) {
#pragma unroll
      for (int c = 0; c < K; c += 4) {
        uint4 v;
        v.x = conv<G, F32>(g.next());
        v.y = conv<G, F32>(g.next());
        v.z = conv<G, F32>(g.next());
        v.w = conv<G, F32>(g.next());
        *reinterpret_cast<uint4*>(my + c) = v;
      }
    } else {
      for (int c = 0; c < w; c++) my[c] = conv<G, F32>(g.next());
    }
    __syncthreads();
    if (w == K && vec_ok && last_row * d.pitch + c0 + K <= d.limit) {
      constexpr int CH = K / 4;  // 16-byte chunks per row
      for (int i = tid; i < T * CH; i += T) {
        const int r = i / CH, ch = i % CH;
        const uint64_t rr = row0 + r;
        if (rr < d.n_rows)
          st_out4(out + rr * d.pitch + c0 + 4 * ch,
                  *reinterpret_cast<const uint4*>(t + r * SP + 4 * ch));
      }
    } else {
      copy_rows_scalar<T>(t, SP, out, d.pitch, row0, d.n_rows, c0, w, d.limit);
    }
    buf ^= 1;
  }
  if (active && !d.jump) g.store(d.state, d.n_rows, row);
}

// Skip without output for XOR128 (plain stepping).
template <class G>
__global__ void k_skip_step(const FillDesc d) {
  const uint64_t row = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= d.n_rows) return;
  G g;
  g.load(d.state, d.n_rows, row);
  for (uint64_t k = 0; k < d.n_per; k++) g.next();
  g.store(d.state, d.n_rows, row);
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

template <class G, int T, int K, bool F32>
static cudaError_t launch_tkf(const FillDesc& d, cudaStream_t s) {
  constexpr size_t bytes = 2ull * T * (K + 4) * sizeof(uint32_t);
  static bool configured = false;  // attribute set once per instantiation
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_fill_simple<G, T, K, F32>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const uint64_t grid = (d.n_rows + T - 1) / T;
  k_fill_simple<G, T, K, F32><<<(unsigned)grid, T, bytes, s>>>(d);
  return cudaGetLastError();
}

template <class G, int T, int K>
static cudaError_t launch_tk(const FillDesc& d, cudaStream_t s) {
  return d.f32 ? launch_tkf<G, T, K, true>(d, s) : launch_tkf<G, T, K, false>(d, s);
}

template <class G>
static cudaError_t launch_g(const FillDesc& d, Tile t, cudaStream_t s) {
  if (t.threads == 64 && t.cols == 32) return launch_tk<G, 64, 32>(d, s);
  if (t.threads == 64 && t.cols == 64) return launch_tk<G, 64, 64>(d, s);
  if (t.threads == 256 && t.cols == 32) return launch_tk<G, 256, 32>(d, s);
  if (t.threads == 128 && t.cols == 64) return launch_tk<G, 128, 64>(d, s);
  return launch_tk<G, 128, 32>(d, s);
}

cudaError_t launch_fill_simple(int gen, const FillDesc& d, Tile t, cudaStream_t s) {
  if (d.n_rows == 0 || d.n_per == 0) return cudaSuccess;
  if (d.out == nullptr) {  // skip
    if (gen == XOR128) {
      k_skip_step<Xor128Gen><<<(unsigned)((d.n_rows + 127) / 128), 128, 0, s>>>(d);
      return cudaGetLastError();
    }
    return launch_skip_mlcg(gen, d.state, d.n_rows, d.n_per, s);
  }
  switch (gen) {
    case GGL: return launch_g<GglGen>(d, t, s);
    case XOR128: return launch_g<Xor128Gen>(d, t, s);
    case RANECU: return launch_g<RanecuGen>(d, t, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_skip_mlcg(int gen, uint32_t* state, uint64_t n, uint64_t k, cudaStream_t s) {
  if (n == 0 || k == 0) return cudaSuccess;
  k_skip_mlcg<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(gen, state, n, k);
  return cudaGetLastError();
}

}  // namespace prng
