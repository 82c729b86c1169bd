// batch.cuh -- descriptors and work-queue helpers of the batched fill.
//
// A batch is a set of fills of distinct handles run as one pass: every
// request is cut into work items (a range of its streams), the items of one
// generator family sit in one array, longest first, and a persistent kernel
// per family pops them with an atomic counter until the array is used up.
// Nothing waits on anything: a block that pops an index past the end exits.
#pragma once

#include "common.cuh"

namespace prng {

// One request as the kernels see it: the fill descriptor of the handle's
// pass (pitch = n_per, limit = n_valid, pos = start position), plus the
// re-seeding fields.
struct BatchReq {
  FillDesc d;
  uint64_t seed;       // re-seed base (if reseed)
  int32_t gen, reseed;
};

// Rows [row0, row0 + rows) of request req.
struct BatchItem {
  uint32_t req;
  uint32_t rows;
  uint64_t row0;
};

// Families, each with its own item array and counter.  Fills are split by
// output type as well (the float form of a family is kind + FAM_F32).
enum BatchFamily : int {
  FAM_SEED = 0, FAM_MLCG, FAM_XOR128, FAM_RANMAR, FAM_MT,
  FAM_LUX24, FAM_LUX48, FAM_LUX97, FAM_LUX223, FAM_LUX389, FAM_KINDS,
  FAM_F32 = FAM_KINDS - 1,
  FAM_COUNT = 2 * FAM_KINDS - 1
};

struct BatchQueue {
  const BatchReq* reqs;
  const BatchItem* items;
  uint32_t n_items;
  uint32_t* counter;   // work counter, zeroed before each pass
};

__device__ __forceinline__ const FillDesc& batch_desc(const BatchReq& r) { return r.d; }

// CTA-wide pop: the same item index for every thread of the block.
__device__ __forceinline__ uint32_t pop_cta(uint32_t* counter, uint32_t* slot) {
  __syncthreads();
  if (threadIdx.x == 0) *slot = atomicAdd(counter, 1u);
  __syncthreads();
  return *slot;
}

// Warp-wide pop.
__device__ __forceinline__ uint32_t pop_warp(uint32_t* counter) {
  uint32_t v = 0;
  if ((threadIdx.x & 31) == 0) v = atomicAdd(counter, 1u);
  return __shfl_sync(0xFFFFFFFFu, v, 0);
}


// Launchers of the persistent family kernels (grid = resident capacity).
cudaError_t launch_batch_seed(const BatchQueue& q, cudaStream_t s);
cudaError_t launch_batch_mlcg(const BatchQueue& q, Tile t, cudaStream_t s);
cudaError_t launch_batch_xor128(const BatchQueue& q, Tile t, bool f32, cudaStream_t s);
cudaError_t launch_batch_ranmar(const BatchQueue& q, Tile t, bool f32, cudaStream_t s);
cudaError_t launch_batch_mt(const BatchQueue& q, Tile t, bool f32, cudaStream_t s);
cudaError_t launch_batch_ranlux(const BatchQueue& q, int p, Tile t, bool f32, cudaStream_t s);

int sm_count();

}  // namespace prng
