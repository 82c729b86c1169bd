// k_simple.cu -- staged bulk fill of the register-state generators XOR128
// (Section 3.3), which has no cheap jump-ahead, and GGL (Section 3.2) and
// RANECU (Section 3.4), whose fills can also run lane-parallel (k_mlcg.cu;
// the launch tile selects which).
//
// One thread owns one stream (or one jump chunk) with its state in
// registers.  Output is stream-major, so a warp's 32 streams write 32
// different rows: each thread drafts K consecutive draws into its row of a
// shared-memory tile with 16-byte stores, then the CTA writes the tile out
// row by row (each 16-byte store instruction of a warp covers whole
// 128-byte runs of rows),
// which turns the per-thread sequences into coalesced HBM writes.  With S = 2
// tiles one barrier per tile suffices; S = 1 halves the shared memory per
// stream (two barriers per tile) so that every stream of a large handle can
// be resident at once instead of running a partial second wave.
#include "batch.cuh"

namespace prng {

struct GglGen {
  static constexpr int SH = 7, WB = 31;
  static constexpr bool JUMPS = true;
  uint32_t x;
  // Row of a jump fill: x0 a^k mod m (Appendix A, eq. MLCG).
  __device__ __forceinline__ void jump_start(uint64_t x0, uint64_t k) {
    x = mulmod_pm<1u>(powmod_pm<1u>(16807u, k), (uint32_t)x0);
  }
  __device__ __forceinline__ void load(const uint32_t* st, uint64_t n, uint64_t row) { x = st[row]; }
  __device__ __forceinline__ void store(uint32_t* st, uint64_t n, uint64_t row) const { st[row] = x; }
  __device__ __forceinline__ void zero() { x = 1; }
  // x <- 16807 x mod (2^31 - 1)  (Section 3.2 constants).
  __device__ __forceinline__ uint32_t next() {
    x = mlcg_step<16807u, 1u>(x);
    return x;
  }
};

struct RanecuGen {
  static constexpr int SH = 7, WB = 31;
  static constexpr bool JUMPS = true;
  uint32_t s1, s2;
  // Row of a jump fill: each component jumped separately from x0 = s1 | s2 << 32.
  __device__ __forceinline__ void jump_start(uint64_t x0, uint64_t k) {
    s1 = mulmod_pm<85u>(powmod_pm<85u>(40014u, k), (uint32_t)(x0 & 0xFFFFFFFFu));
    s2 = mulmod_pm<249u>(powmod_pm<249u>(40692u, k), (uint32_t)(x0 >> 32));
  }
  __device__ __forceinline__ void load(const uint32_t* st, uint64_t n, uint64_t row) {
    s1 = st[row];
    s2 = st[n + row];
  }
  __device__ __forceinline__ void store(uint32_t* st, uint64_t n, uint64_t row) const {
    st[row] = s1;
    st[n + row] = s2;
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

struct Xor128Gen {
  static constexpr int SH = 8, WB = 32;
  static constexpr bool JUMPS = false;
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

template <class G, int OM>
__device__ __forceinline__ uint32_t conv(uint32_t v) {
  if constexpr (OM == OUT_F32) return as_f32_bits<G::SH>(v);
  else return v;   // u32, or a raw draw paired at the copy-out
}

// Row-major tile, thread t's K staged draws in row t.  16-byte chunk ch of
// row t is stored at chunk slot ch ^ (t & 7): eight consecutive threads
// writing the same chunk, or eight lanes reading eight chunks of one row,
// touch eight different bank quads, without padding the rows.
template <int K>
__device__ __forceinline__ int swz(int row, int ch) { return ch ^ (row & 7); }

// Streams [row0, row0 + T) of a fill, one per thread; smem holds S tiles of
// T * K words.
template <class G, int T, int K, int S, int OM>
__device__ __forceinline__ void simple_rows(const FillDesc& d, uint64_t row0, uint32_t* smem) {
  static_assert(K % 32 == 0, "tile rows hold whole 8-chunk swizzle groups");
  constexpr int CH = K / 4;          // 16-byte chunks per row
  constexpr int RS = T / CH;         // rows one copy-out pass of the CTA covers
  static_assert(RS % 8 == 0, "copy-out rows of one thread must share a swizzle phase");
  const int tid = threadIdx.x;
  const uint64_t row = row0 + tid;
  const bool active = row < d.n_rows;

  G g;
  if (!active) {
    g.zero();
  } else if constexpr (G::JUMPS) {
    if (d.jump) g.jump_start(d.x0, row * d.pitch);   // chunk `row` of one sequence
    else g.load(d.state, d.n_rows, row);
  } else {
    g.load(d.state, d.n_rows, row);
  }

  uint32_t* out = static_cast<uint32_t*>(d.out);
  const bool vec_ok = ((d.pitch & 3) == 0) && ((reinterpret_cast<uintptr_t>(out) & 15) == 0);
  // Copy-out role of this thread: chunk `cch` of rows cr0 + RS k, k < CH.
  const int cch = tid % CH, cr0 = tid / CH;
  const int cslot = swz<K>(cr0, cch);           // (cr0 + RS k) & 7 == cr0 & 7
  uint32_t* cg = out + (row0 + cr0) * d.pitch + 4 * cch;
  const uint64_t cstep = (uint64_t)RS * d.pitch;
  const uint64_t left = d.n_rows > row0 + cr0 ? d.n_rows - (row0 + cr0) : 0;
  const int crows = left >= (uint64_t)RS * (CH - 1) + 1 ? CH : (int)((left + RS - 1) / RS);
  const uint64_t last_row = (row0 + T < d.n_rows ? row0 + T : d.n_rows) - 1;
  const int sw = tid & 7;

  const uint64_t n = d.n_per;
  int buf = 0;
  for (uint64_t c0 = 0; c0 < n; c0 += K) {
    const int w = (n - c0 < (uint64_t)K) ? (int)(n - c0) : K;
    uint32_t* const t = smem + buf * (T * K);
    uint32_t* my = t + tid * K;
    if (w == K) {
#pragma unroll
      for (int c = 0; c < CH; c++) {
        uint4 v;
        v.x = conv<G, OM>(g.next());
        v.y = conv<G, OM>(g.next());
        v.z = conv<G, OM>(g.next());
        v.w = conv<G, OM>(g.next());
        *reinterpret_cast<uint4*>(my + 4 * (c ^ sw)) = v;
      }
    } else {
      for (int c = 0; c < w; c++) my[4 * ((c >> 2) ^ sw) + (c & 3)] = conv<G, OM>(g.next());
    }
    __syncthreads();
    if (w == K && (vec_ok || OM == OUT_ISING) && last_row * d.pitch + c0 + K <= d.limit) {
      const uint32_t* src = t + cr0 * K + 4 * cslot;
      uint32_t* dst = cg + c0;
      const uint64_t edst = (row0 + cr0) * d.pitch + 4 * cch + c0;
#pragma unroll
      for (int k = 0; k < CH; k++)
        if (k < crows) {
          if constexpr (OM == OUT_ISING)
            put4<OM, G::WB>(d, nullptr, edst + k * cstep, *reinterpret_cast<const uint4*>(src + k * RS * K));
          else
            st_chunk<OM, G::WB>(dst + k * cstep, *reinterpret_cast<const uint4*>(src + k * RS * K));
        }
    } else {
      // Partial tile, unaligned output or a jump fill's last chunk: scalar
      // stores, warp per row, lanes on consecutive columns.
      constexpr int NW = T / 32;
      const int lane = tid & 31, wi = tid >> 5;
      for (int r = wi; r < T; r += NW) {
        const uint64_t rr = row0 + r;
        if (rr >= d.n_rows) break;
        const uint64_t base = rr * d.pitch + c0;
        if constexpr (OM == OUT_F64) {   // w, base and the limit are even
          for (int c = 2 * lane; c < w; c += 64)
            if (base + c < d.limit)
              st_pair<G::WB>(out + base + c, t[r * K + 4 * ((c >> 2) ^ (r & 7)) + (c & 3)],
                             t[r * K + 4 * ((c >> 2) ^ (r & 7)) + (c & 3) + 1]);
        } else {
          for (int c = lane; c < w; c += 32)
            if (base + c < d.limit)
              put1<OM>(d, out + base + c, base + c, t[r * K + 4 * ((c >> 2) ^ (r & 7)) + (c & 3)]);
        }
      }
    }
    if constexpr (S == 1) __syncthreads();
    else buf ^= 1;
  }
  if (active && !d.jump) g.store(d.state, d.n_rows, row);
}

template <class G, int T, int K, int S, int OM>
__global__ void __launch_bounds__(T) k_fill_simple(const FillDesc d) {
  extern __shared__ __align__(16) uint32_t smem[];
  simple_rows<G, T, K, S, OM>(d, (uint64_t)blockIdx.x * T, smem);
}

// Batched XOR128 fills: a block pops an item (T streams of one request).
template <int T, int K, int S, bool F32>
__global__ void __launch_bounds__(T) k_batch_xor128(const BatchQueue q) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ uint32_t slot;
  for (;;) {
    const uint32_t it = pop_cta(q.counter, &slot);
    if (it >= q.n_items) break;
    const BatchItem si = q.items[it];
    __shared__ FillDesc sd;
    load_desc(&sd, q.reqs[si.req].d, threadIdx.x, T);
    __syncthreads();
    simple_rows<Xor128Gen, T, K, S, F32 ? OUT_F32 : OUT_U32>(sd, si.row0, smem);
  }
}

template <int T, int K, int S, bool F32>
static cudaError_t launch_bx(const BatchQueue& q, cudaStream_t s) {
  constexpr size_t bytes = (size_t)S * T * K * sizeof(uint32_t);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_batch_xor128<T, K, S, F32>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_xor128<T, K, S, F32>, T, bytes);
  const uint32_t cap = (uint32_t)sm_count() * (per_sm > 0 ? per_sm : 1);
  k_batch_xor128<T, K, S, F32><<<q.n_items < cap ? q.n_items : cap, T, bytes, s>>>(q);
  return cudaGetLastError();
}

template <int T, int K, int S>
static cudaError_t launch_bx2(const BatchQueue& q, bool f32, cudaStream_t s) {
  return f32 ? launch_bx<T, K, S, true>(q, s) : launch_bx<T, K, S, false>(q, s);
}

cudaError_t launch_batch_xor128(const BatchQueue& q, Tile t, bool f32, cudaStream_t s) {
  if (q.n_items == 0) return cudaSuccess;
  if (t.threads == 64 && t.cols == 32 && t.stages == 1) return launch_bx2<64, 32, 1>(q, f32, s);
  if (t.threads == 128 && t.cols == 32 && t.stages == 2) return launch_bx2<128, 32, 2>(q, f32, s);
  if (t.threads == 128 && t.cols == 64 && t.stages == 1) return launch_bx2<128, 64, 1>(q, f32, s);
  if (t.threads == 256 && t.cols == 32 && t.stages == 1) return launch_bx2<256, 32, 1>(q, f32, s);
  return launch_bx2<128, 32, 1>(q, f32, s);
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

template <class G, int T, int K, int S, int OM>
static cudaError_t launch_tkf(const FillDesc& d, cudaStream_t s) {
  constexpr size_t bytes = (size_t)S * T * K * sizeof(uint32_t);
  static bool configured = false;  // attribute set once per instantiation
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_fill_simple<G, T, K, S, OM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const uint64_t grid = (d.n_rows + T - 1) / T;
  k_fill_simple<G, T, K, S, OM><<<(unsigned)grid, T, bytes, s>>>(d);
  return cudaGetLastError();
}

template <class G, int T, int K, int S>
static cudaError_t launch_tk(const FillDesc& d, cudaStream_t s) {
  return with_mode(d.mode, [&](auto m) { return launch_tkf<G, T, K, S, decltype(m)::value>(d, s); });
}

// Supported tiles: (threads, cols, stages).
template <class G>
static cudaError_t launch_g(const FillDesc& d, Tile t, cudaStream_t s) {
  if (t.threads == 128 && t.cols == 32 && t.stages == 2) return launch_tk<G, 128, 32, 2>(d, s);
  if (t.threads == 128 && t.cols == 64 && t.stages == 1) return launch_tk<G, 128, 64, 1>(d, s);
  if (t.threads == 256 && t.cols == 32 && t.stages == 1) return launch_tk<G, 256, 32, 1>(d, s);
  return launch_tk<G, 128, 32, 1>(d, s);
}

cudaError_t launch_fill_simple(int gen, const FillDesc& d, Tile t, cudaStream_t s) {
  if (d.n_rows == 0 || d.n_per == 0) return cudaSuccess;
  if (d.out == nullptr) {  // skip: plain stepping (the MLCG generators jump instead)
    if (gen != XOR128) return cudaErrorInvalidValue;
    k_skip_step<Xor128Gen><<<(unsigned)((d.n_rows + 127) / 128), 128, 0, s>>>(d);
    return cudaGetLastError();
  }
  switch (gen) {
    case GGL: return launch_g<GglGen>(d, t, s);
    case XOR128: return launch_g<Xor128Gen>(d, t, s);
    case RANECU: return launch_g<RanecuGen>(d, t, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace prng
