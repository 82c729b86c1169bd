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
  constexpr uint64_t per_block = (uint64_t)kIsingThreads * kIsingSitesPerThread;
  for (uint32_t first = 0; first < n; first += kIsingPerLaunch) {
    IsingLaunch b;
    b.n = n - first < (uint32_t)kIsingPerLaunch ? n - first : (uint32_t)kIsingPerLaunch;
    uint64_t blocks = 0;
    for (uint32_t i = 0; i < b.n; i++) {
      b.r[i] = reqs[first + i];
      b.block0[i] = (uint32_t)blocks;
      const uint64_t sites = (uint64_t)b.r[i].L * (b.r[i].L / 2);
      blocks += (sites + per_block - 1) / per_block;
    }
    if (blocks > 0x7FFFFFFFull) return PRNG_ESIZE;
    b.block0[b.n] = (uint32_t)blocks;
    k_ising_half_sweep<<<(unsigned)blocks, kIsingThreads, 0, s>>>(b);
    if (cudaGetLastError() != cudaSuccess) return PRNG_ECUDA;
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
