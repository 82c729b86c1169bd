// k_seed.cu -- on-device seeding of every stream of a handle (the paper
// initialises its lag tables on the GPU too, Section 3.1).
//
// Stream i takes s = splitmix64(seed + i) and maps it into its generator's
// seed range, then runs the generator's own table initialisation:
//   GGL      x0 = 1 + s mod (2^31 - 2)
//   XOR128   (x, y, z, w) = 32-bit halves of s and of splitmix64(s)
//   RANECU   s1 = 1 + lo32(s) mod (m1 - 1), s2 = 1 + hi32(s) mod (m2 - 1)
//   RANMAR   RMARIN(ij = lo32(s) mod 31329, kl = hi32(s) mod 30082)
//   RANLUX   24 words from the MLCG 40014 mod 2147483563 started at
//            s mod 2147483563 (19780503 when that is 0), carry = (x_{-1} == 0)
//   MT19937  init_genrand(lo32(s))
//
// Also the host helpers the launchers share: the SM count, and the
// retained stream-ordered scratch pool of the jump fills.
#include <mutex>

#include "batch.cuh"
#include "scratch.cuh"

namespace prng {

// RMARIN (James 1988, cited by Section 3.5): 97 entries of 24 bits, most
// significant bit first, from the lagged product generator mod 179 and the
// LCG (53 l + 1) mod 169.  Written in canonical order V[k] = U[97 - k].
__device__ void rmarin_to_state(uint32_t ij, uint32_t kl, uint32_t* st, uint64_t n, uint64_t row) {
  uint32_t i = (ij / 177) % 177 + 2, j = ij % 177 + 2;
  uint32_t k = (kl / 169) % 178 + 1, l = kl % 169;
  for (int ii = 1; ii <= 97; ii++) {
    uint32_t acc = 0;
    for (int b = 23; b >= 0; b--) {
      const uint32_t m = ((i * j) % 179 * k) % 179;
      i = j;
      j = k;
      k = m;
      l = (53 * l + 1) % 169;
      acc |= ((l * m) % 64 >= 32 ? 1u : 0u) << b;
    }
    st[(uint64_t)(97 - ii) * n + row] = acc;
  }
  st[97 * n + row] = 362436u;  // C_0 = 362436 / 2^24
}

// Seed stream `row` of a handle of n streams (state layout in common.cuh).
__device__ void seed_stream(int gen, uint64_t seed, uint64_t n, uint32_t* st, uint64_t row) {
  const uint64_t s = splitmix64(seed + row);
  const uint32_t lo = (uint32_t)s, hi = (uint32_t)(s >> 32);
  switch (gen) {
    case GGL:
      st[row] = (uint32_t)(1 + s % 2147483646ull);
      break;
    case XOR128: {
      const uint64_t t = splitmix64(s);
      uint32_t z = (uint32_t)t, w = (uint32_t)(t >> 32);
      if ((lo | hi | z | w) == 0) w = 1;
      st[row] = lo;
      st[n + row] = hi;
      st[2 * n + row] = z;
      st[3 * n + row] = w;
      break;
    }
    case RANECU:
      st[row] = 1 + lo % 2147483562u;
      st[n + row] = 1 + hi % 2147483398u;
      break;
    case RANMAR:
      rmarin_to_state(lo % 31329u, hi % 30082u, st, n, row);
      break;
    case RANLUX: {
      uint32_t x = (uint32_t)(s % 2147483563ull);
      if (x == 0) x = 19780503u;
      uint32_t last = 0;
      for (int k = 0; k < 24; k++) {
        x = mlcg_step<40014u, 85u>(x);
        last = x & 0xFFFFFFu;
        st[(uint64_t)k * n + row] = last;
      }
      st[24 * n + row] = (last == 0) ? 1u : 0u;
      break;
    }
    case MT19937: {
      uint32_t* mt = st + row * 624;
      uint32_t v = lo;
      mt[0] = v;
      for (uint32_t k = 1; k < 624; k++) {
        v = 1812433253u * (v ^ (v >> 30)) + k;
        mt[k] = v;
      }
      break;
    }
  }
}

__global__ void k_seed(int gen, uint64_t seed, uint64_t n, uint32_t* st) {
  const uint64_t row = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row < n) seed_stream(gen, seed, n, st, row);
}

// Persistent seeding of every re-seeded request of a batch: an item is up
// to 256 consecutive streams of one request.
__global__ void __launch_bounds__(256) k_batch_seed(const BatchQueue q) {
  __shared__ uint32_t slot;
  for (;;) {
    const uint32_t it = pop_cta(q.counter, &slot);
    if (it >= q.n_items) break;
    const BatchItem I = q.items[it];
    const BatchReq& r = q.reqs[I.req];
    if (threadIdx.x < I.rows) seed_stream(r.gen, r.seed, r.d.n_rows, r.d.state, I.row0 + threadIdx.x);
  }
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    n = (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0) ? v : 1;
  }
  return n;
}

namespace {
constexpr int kMaxPoolDevices = 64;
std::mutex g_pool_lock;
cudaMemPool_t g_pool[kMaxPoolDevices] = {};
}  // namespace

cudaError_t scratch_alloc(void** p, size_t bytes, cudaStream_t s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxPoolDevices) return cudaErrorInvalidDevice;
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> guard(g_pool_lock);
    if (g_pool[dev] == nullptr) {
      cudaMemPoolProps props{};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      e = cudaMemPoolCreate(&pool, &props);
      if (e != cudaSuccess) return e;
      uint64_t keep = UINT64_MAX;   // never trim: freed blocks stay for the next call
      e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      if (e != cudaSuccess) {
        cudaMemPoolDestroy(pool);
        return e;
      }
      g_pool[dev] = pool;
    }
    pool = g_pool[dev];
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

cudaError_t scratch_free(void* p, cudaStream_t s) { return cudaFreeAsync(p, s); }

cudaError_t launch_batch_seed(const BatchQueue& q, cudaStream_t s) {
  if (q.n_items == 0) return cudaSuccess;
  const uint32_t cap = (uint32_t)sm_count() * 8;
  k_batch_seed<<<q.n_items < cap ? q.n_items : cap, 256, 0, s>>>(q);
  return cudaGetLastError();
}

cudaError_t launch_seed(int gen, int p, uint64_t seed, uint64_t n, uint32_t* state, cudaStream_t s) {
  (void)p;
  if (n == 0) return cudaSuccess;
  const int T = (gen == RANMAR || gen == MT19937) ? 64 : 256;
  k_seed<<<(unsigned)((n + T - 1) / T), T, 0, s>>>(gen, seed, n, state);
  return cudaGetLastError();
}

}  // namespace prng
