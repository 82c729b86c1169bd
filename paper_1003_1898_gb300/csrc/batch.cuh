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
// RANLUX has one family per luxury p (the p is a kernel template argument).
enum BatchFamily : int {
  FAM_SEED = 0, FAM_MLCG, FAM_XOR128, FAM_RANMAR, FAM_MT,
  FAM_LUX24, FAM_LUX48, FAM_LUX97, FAM_LUX223, FAM_LUX389,
  FAM_LUX120, FAM_LUX240, FAM_LUX408, FAM_KINDS,
  FAM_F32 = FAM_KINDS - 1,
  FAM_COUNT = 2 * FAM_KINDS - 1
};

// The luxury p of each RANLUX family, in family order from FAM_LUX24.
constexpr int kLuxFamilyP[FAM_KINDS - FAM_LUX24] = {24, 48, 97, 223, 389, 120, 240, 408};

inline int family_of(int gen, int p) {
  switch (gen) {
    case GGL:
    case RANECU: return FAM_MLCG;
    case XOR128: return FAM_XOR128;
    case RANMAR: return FAM_RANMAR;
    case MT19937: return FAM_MT;
    default:
      for (int i = 0; i < FAM_KINDS - FAM_LUX24; i++)
        if (kLuxFamilyP[i] == p) return FAM_LUX24 + i;
      return -1;
  }
}
// Family of a fill (the MLCG kernel takes the output type at run time).
inline int fill_family(int gen, int p, bool f32) {
  const int kind = family_of(gen, p);
  return (f32 && kind != FAM_MLCG) ? kind + FAM_F32 : kind;
}
inline int kind_of(int fam) { return fam >= FAM_KINDS ? fam - FAM_F32 : fam; }
inline bool is_f32_family(int fam) { return fam >= FAM_KINDS; }
inline int lux_p_of(int fam) { return kLuxFamilyP[kind_of(fam) - FAM_LUX24]; }

// Launch tile of a family.  RANLUX takes 32-thread CTAs here rather than its
// bulk-fill tile: a work item is one CTA's rows of one request, and most
// requests of a batch have few streams, so 32-row items waste fewer threads
// (measured: 0.75 against 0.50 numbers/ns with 64-row items on the mixed
// 20,000-request batch).  The others use the generator's default tile.
inline Tile tile_of(int fam) {
  const int k = kind_of(fam);
  if (k == FAM_SEED) return Tile{256, 0, 1};
  if (k >= FAM_LUX24) return Tile{32, 48, 1};
  const int gen = k == FAM_MLCG ? GGL : k == FAM_XOR128 ? XOR128 : k == FAM_RANMAR ? RANMAR : MT19937;
  return default_tile(gen, 0);
}

// Streams per work item of a family launched with tile t.
inline uint32_t rows_per_item(int fam, Tile t) {
  switch (kind_of(fam)) {
    case FAM_SEED: return 256;
    case FAM_MLCG: return 4;
    case FAM_MT: return 2;
    case FAM_RANMAR: return (uint32_t)t.threads / 32;  // a warp per stream
    default: return (uint32_t)t.threads;
  }
}

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

// The descriptor of a work item, copied into shared memory by the threads
// [0, NT) that share it (then synchronised by the caller): the kernels then
// read it from shared memory, which their global stores cannot alias, so its
// fields stay in registers instead of being reloaded after every store.
__device__ __forceinline__ void load_desc(FillDesc* dst, const FillDesc& src, int t, int nt) {
  static_assert(sizeof(FillDesc) % 4 == 0, "descriptor copied as words");
  const uint32_t* s = reinterpret_cast<const uint32_t*>(&src);
  uint32_t* d = reinterpret_cast<uint32_t*>(dst);
  for (int i = t; i < (int)(sizeof(FillDesc) / 4); i += nt) d[i] = s[i];
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
