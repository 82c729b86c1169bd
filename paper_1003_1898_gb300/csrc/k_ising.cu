// k_ising.cu -- checkerboard Metropolis half-sweeps of 2-D Ising lattices
// that consume the generators' draws (the Monte Carlo use the paper's
// generators serve; Section 3.5 cites RANMAR's earlier Ising simulations).
//
// Periodic L x L lattice, J = 1, h = 0, spins +1/-1 in int8, row-major.  A
// half-sweep visits the sites of one colour ((x + y) % 2); sites of one
// colour only neighbour the other colour, so they update independently.
// The site with colour rank k (k = y L/2 + x/2) takes draw k, whose 24-bit
// value r = draw >> shift decides the proposal with integer thresholds:
// accept when dE = 2 s (sum of neighbours) <= 0, or r < t4 (dE = 4), or
// r < t8 (dE = 8).  Thresholds are computed once on the host, so both the
// library and any checker take the same integer decision.
//
// Up to kIsingPerLaunch lattices go to one launch with their descriptors
// passed by value; a block works on one lattice (block ranges by prefix).
// Lattices whose rows split into 16-byte chunks (L a multiple of 16, both
// buffers 16-byte aligned, and a draw layout that keeps 8 consecutive
// ranks in one row) take the vector form: a thread owns 16 consecutive
// sites of a row, 8 of them of the colour, and moves them as one 16-byte
// load and store per row (its own row and the rows above and below) and two
// 16-byte draw loads.  The others take the scalar form, a thread per site.
#include <cmath>

#include "../../include/prng.h"
#include "common.cuh"

namespace prng {

constexpr int kIsingPerLaunch = 96;
constexpr int kIsingThreads = 256;
constexpr int kIsingSitesPerThread = 4;

struct IsingLaunch {
  prng_ising_req r[kIsingPerLaunch];
  uint32_t block0[kIsingPerLaunch + 1];  // first block of each lattice
  uint32_t n;
};

__global__ void __launch_bounds__(kIsingThreads) k_ising_half_sweep(const __grid_constant__ IsingLaunch b) {
  // Lattice of this block: largest i with block0[i] <= blockIdx.x.
  uint32_t lo = 0, hi = b.n;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (b.block0[mid] <= blockIdx.x) lo = mid;
    else hi = mid;
  }
  const prng_ising_req& q = b.r[lo];
  const uint32_t L = q.L, half = L >> 1;
  const uint64_t sites = (uint64_t)L * half;
  const uint64_t base = (uint64_t)(blockIdx.x - b.block0[lo]) * kIsingThreads * kIsingSitesPerThread;
#pragma unroll
  for (int j = 0; j < kIsingSitesPerThread; j++) {
    const uint64_t k = base + (uint64_t)j * kIsingThreads + threadIdx.x;
    if (k >= sites) break;
    const uint32_t y = (uint32_t)(k / half);
    const uint32_t x = 2 * (uint32_t)(k - (uint64_t)y * half) + ((y + q.colour) & 1u);
    const uint32_t yu = y == 0 ? L - 1 : y - 1, yd = y + 1 == L ? 0 : y + 1;
    const uint32_t xl = x == 0 ? L - 1 : x - 1, xr = x + 1 == L ? 0 : x + 1;
    int8_t* row = q.d_spins + (uint64_t)y * L;
    const int s = row[x];
    const int nb = q.d_spins[(uint64_t)yu * L + x] + q.d_spins[(uint64_t)yd * L + x] + row[xl] + row[xr];
    const int dE = 2 * s * nb;
    uint64_t di = k;
    if (q.pitch != 0) {   // k < 2^31: 32-bit quotient, a shift when per is a power of two
      const uint32_t k32 = (uint32_t)k, per = q.per;
      const uint32_t row = (per & (per - 1)) == 0 ? k32 >> (__ffs(per) - 1) : k32 / per;
      di = (uint64_t)row * q.pitch + (k32 - row * per);
    }
    const uint32_t r = q.d_draws[di] >> q.shift;
    const bool accept = dE <= 0 || (dE == 4 ? r < q.t4 : r < q.t8);
    if (accept) row[x] = (int8_t)(-s);
  }
}

// Vector form.  The 16-byte store also rewrites the 8 sites of the other
// colour with the values it read: nothing changes them during the
// half-sweep, so readers of those neighbours see the same bytes.
constexpr int kIsingVecThreads = 256;

__device__ __forceinline__ uint32_t ising_lattice_of(const IsingLaunch& b) {
  uint32_t lo = 0, hi = b.n;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (b.block0[mid] <= blockIdx.x) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(kIsingVecThreads) k_ising_half_sweep_v(const __grid_constant__ IsingLaunch b) {
  const uint32_t lo = ising_lattice_of(b);
  const prng_ising_req& q = b.r[lo];
  const uint32_t L = q.L, cpr = L >> 4;                      // 16-site chunks per row
  const uint32_t chunk = (blockIdx.x - b.block0[lo]) * kIsingVecThreads + threadIdx.x;
  if (chunk >= L * cpr) return;                              // L <= 65534: L * L / 16 < 2^28
  const uint32_t y = chunk / cpr, x0 = (chunk - y * cpr) << 4;
  const uint32_t yu = y == 0 ? L - 1 : y - 1, yd = y + 1 == L ? 0 : y + 1;
  int8_t* row = q.d_spins + (uint64_t)y * L;
  union V { uint4 v; int8_t c[16]; };
  V C, U, D;
  C.v = *reinterpret_cast<const uint4*>(row + x0);
  U.v = *reinterpret_cast<const uint4*>(q.d_spins + (uint64_t)yu * L + x0);
  D.v = *reinterpret_cast<const uint4*>(q.d_spins + (uint64_t)yd * L + x0);
  const int lft = row[x0 == 0 ? L - 1 : x0 - 1];
  const int rgt = row[x0 + 16 == L ? 0 : x0 + 16];
  const uint32_t par = (y + q.colour) & 1u;                 // x parity of the colour in row y
  const uint32_t k0 = y * (L >> 1) + (x0 >> 1);              // colour rank of the first site
  uint64_t di = k0;
  if (q.pitch != 0) {   // 8 ranks never straddle a row of `per` (per % 8 == 0)
    const uint32_t per = q.per;
    const uint32_t pr = (per & (per - 1)) == 0 ? k0 >> (__ffs(per) - 1) : k0 / per;
    di = (uint64_t)pr * q.pitch + (k0 - pr * per);
  }
  const uint4 d0 = *reinterpret_cast<const uint4*>(q.d_draws + di);
  const uint4 d1 = *reinterpret_cast<const uint4*>(q.d_draws + di + 4);
  const uint32_t dr[8] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
  V O = C;
#pragma unroll
  for (int i = 0; i < 8; i++) {
#pragma unroll
    for (int p = 0; p < 2; p++) {     // compile-time byte index for each parity
      if ((uint32_t)p != par) continue;
      const int bi = 2 * i + p;
      const int s = C.c[bi];
      const int l = bi == 0 ? lft : C.c[bi - 1];
      const int r = bi == 15 ? rgt : C.c[bi + 1];
      const int dE = 2 * s * (U.c[bi] + D.c[bi] + l + r);
      const uint32_t v = dr[i] >> q.shift;
      const bool accept = dE <= 0 || (dE == 4 ? v < q.t4 : v < q.t8);
      if (accept) O.c[bi] = (int8_t)(-s);
    }
  }
  *reinterpret_cast<uint4*>(row + x0) = O.v;
}

// Whether a lattice can take the vector form.
static bool ising_vec_ok(const prng_ising_req& q) {
  return (q.L & 15u) == 0 && q.L <= 65520 && (reinterpret_cast<uintptr_t>(q.d_spins) & 15) == 0 &&
         (reinterpret_cast<uintptr_t>(q.d_draws) & 15) == 0 &&
         (q.pitch == 0 || ((q.per & 7u) == 0 && (q.pitch & 3u) == 0));
}

}  // namespace prng

using namespace prng;

extern "C" int prng_ising_half_sweep(const prng_ising_req* reqs, uint32_t n, void* stream) {
  if (n == 0) return PRNG_OK;
  if (reqs == nullptr) return PRNG_ENULL;
  for (uint32_t i = 0; i < n; i++) {
    const prng_ising_req& q = reqs[i];
    if (q.d_spins == nullptr || q.d_draws == nullptr) return PRNG_ENULL;
    if (q.L < 2 || (q.L & 1) != 0 || q.colour > 1 || q.shift > 8) return PRNG_ESIZE;
    if (q.pitch != 0 && (q.per == 0 || q.per > q.pitch)) return PRNG_ESIZE;
    if ((reinterpret_cast<uintptr_t>(q.d_draws) & 3) != 0) return PRNG_ESIZE;
  }
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  // Each group of up to kIsingPerLaunch lattices: the vector-form ones in one
  // launch, the rest in another (a thread per 16 sites / per 4 sites).
  for (int vec = 1; vec >= 0; vec--) {
    const uint64_t per_block = vec ? (uint64_t)kIsingVecThreads * 16
                                   : (uint64_t)kIsingThreads * kIsingSitesPerThread * 2;
    IsingLaunch b;
    b.n = 0;
    uint64_t blocks = 0;
    auto flush = [&]() -> bool {
      if (b.n == 0) return true;
      if (blocks > 0x7FFFFFFFull) return false;
      b.block0[b.n] = (uint32_t)blocks;
      if (vec) k_ising_half_sweep_v<<<(unsigned)blocks, kIsingVecThreads, 0, s>>>(b);
      else k_ising_half_sweep<<<(unsigned)blocks, kIsingThreads, 0, s>>>(b);
      b.n = 0;
      blocks = 0;
      return cudaGetLastError() == cudaSuccess;
    };
    for (uint32_t i = 0; i < n; i++) {
      if (ising_vec_ok(reqs[i]) != (vec == 1)) continue;
      b.r[b.n] = reqs[i];
      b.block0[b.n] = (uint32_t)blocks;
      blocks += ((uint64_t)reqs[i].L * reqs[i].L + per_block - 1) / per_block;   // L * L sites
      if (++b.n == (uint32_t)kIsingPerLaunch && !flush()) return blocks > 0x7FFFFFFFull ? PRNG_ESIZE : PRNG_ECUDA;
    }
    if (!flush()) return blocks > 0x7FFFFFFFull ? PRNG_ESIZE : PRNG_ECUDA;
  }
  return PRNG_OK;
}

extern "C" int prng_ising_thresholds(double beta, uint32_t* t4, uint32_t* t8) {
  if (t4 == nullptr || t8 == nullptr) return PRNG_ENULL;
  if (!(beta >= 0.0)) return PRNG_ESIZE;
  *t4 = (uint32_t)std::floor(16777216.0 * std::exp(-4.0 * beta));
  *t8 = (uint32_t)std::floor(16777216.0 * std::exp(-8.0 * beta));
  return PRNG_OK;
}
