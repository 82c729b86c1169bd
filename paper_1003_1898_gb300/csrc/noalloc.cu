// noalloc.cu -- prng_batch_fill_noalloc: the batched fill without any
// memory allocation by the library.
//
// Some callers cannot let a library allocate: code that runs under a
// framework's caching allocator and must not call cudaMalloc behind its
// back, services that reserve all device memory up front, or latency-bound
// loops that cannot afford an allocation (which may synchronise the
// device).  For them this entry point keeps everything the batched pass
// needs besides the caller's handles and outputs -- the per-request
// descriptors, the work items and the work counters -- in one fixed
// file-scope device array, and the host-side staging in a fixed static host
// buffer.  It runs the same family kernels as prng_batch_launch, one after
// the other on the caller's stream.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "../../include/prng.h"
#include "batch.cuh"
#include "handle.cuh"

using namespace prng;

namespace {

constexpr uint32_t kMaxRequests = PRNG_NOALLOC_MAX_REQUESTS;
constexpr uint32_t kMaxItems = PRNG_NOALLOC_MAX_ITEMS;
constexpr size_t kCounterBytes = 256;  // FAM_COUNT work counters, padded
constexpr size_t kReqBytes = kMaxRequests * sizeof(BatchReq);
constexpr size_t kItemBytes = kMaxItems * sizeof(BatchItem);
constexpr size_t kScratchBytes = kCounterBytes + kReqBytes + kItemBytes;
static_assert(FAM_COUNT * sizeof(uint32_t) <= kCounterBytes, "counter area too small");
static_assert(kReqBytes % 16 == 0, "items must stay 16-byte aligned");

// The device scratch: [counters | request descriptors | work items].  Every
// call shares it and it keeps the last call's contents.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Host-side staging of descriptors and items (pageable; a copy from it has
// consumed the source when cudaMemcpyAsync returns).
alignas(256) unsigned char g_host[kReqBytes + kItemBytes];
// The handles of a call, sorted to find duplicates, and their positions
// after the call, committed only once every copy and launch was enqueued.
prng_state* g_sorted[kMaxRequests];
uint32_t g_new_pos[kMaxRequests];
std::mutex g_lock;

// Device address of g_scratch, looked up once per device.
constexpr int kMaxDevices = 64;
unsigned char* g_dev_ptr[kMaxDevices] = {};


}  // namespace

extern "C" int prng_batch_fill_noalloc(const prng_fill_req* reqs, uint32_t n_reqs, void* stream) {
  if (n_reqs == 0) return PRNG_OK;
  if (reqs == nullptr) return PRNG_ENULL;
  if (n_reqs > kMaxRequests) return PRNG_ESCRATCH;
  // The static staging below is shared by every call: host threads take
  // turns from here on.
  std::lock_guard<std::mutex> guard(g_lock);
  // Validate and count items per family (no allocation).
  uint64_t fam_n[FAM_COUNT] = {};
  for (uint32_t i = 0; i < n_reqs; i++) {
    const prng_fill_req& r = reqs[i];
    if (r.st == nullptr) return PRNG_ENULL;
    if (r.n_per_stream > 0 && r.d_out == nullptr) return PRNG_ENULL;
    if ((reinterpret_cast<uintptr_t>(r.d_out) & 3) != 0) return PRNG_ESIZE;
    if (r.n_per_stream > 0 && r.st->n_streams > UINT64_MAX / r.n_per_stream) return PRNG_ESIZE;
    g_sorted[i] = r.st;
    if (r.reseed) fam_n[FAM_SEED] += (r.st->n_streams + 255) / 256;
    if (r.n_per_stream > 0) {
      const int f = fill_family(r.st->gen, r.st->p, r.f32 != 0);
      const uint32_t per = rows_per_item(f, tile_of(f));
      fam_n[f] += (r.st->n_streams + per - 1) / per;
    }
  }
  uint64_t total = 0;
  uint32_t fam_off[FAM_COUNT];
  for (int f = 0; f < FAM_COUNT; f++) {
    fam_off[f] = (uint32_t)std::min<uint64_t>(total, kMaxItems);
    total += fam_n[f];
  }
  if (total > kMaxItems) return PRNG_ESCRATCH;
  // A handle may appear once per call (its streams advance once).
  std::sort(g_sorted, g_sorted + n_reqs);
  if (std::adjacent_find(g_sorted, g_sorted + n_reqs) != g_sorted + n_reqs) return PRNG_EBLOB;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PRNG_ECUDA;
  if (g_dev_ptr[dev] == nullptr) {  // first call on this device: find the array's device address
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return PRNG_ECUDA;
    }
    g_dev_ptr[dev] = static_cast<unsigned char*>(p);
  }
  unsigned char* d_base = g_dev_ptr[dev];
  uint32_t* d_counters = reinterpret_cast<uint32_t*>(d_base);
  BatchReq* d_reqs = reinterpret_cast<BatchReq*>(d_base + kCounterBytes);
  BatchItem* d_items = reinterpret_cast<BatchItem*>(d_base + kCounterBytes + kReqBytes);
  BatchReq* h_reqs = reinterpret_cast<BatchReq*>(g_host);
  BatchItem* h_items = reinterpret_cast<BatchItem*>(g_host + kReqBytes);

  // Descriptors and items; the handles' new positions are kept aside until
  // the whole pass has been enqueued.
  uint32_t fill_at[FAM_COUNT];
  std::memcpy(fill_at, fam_off, sizeof(fill_at));
  for (uint32_t i = 0; i < n_reqs; i++) {
    const prng_fill_req& r = reqs[i];
    prng_state* st = r.st;
    BatchReq& q = h_reqs[i];
    const uint64_t full = st->n_streams * r.n_per_stream;
    std::memset(&q, 0, sizeof(q));
    q.d.state = st->d_state;
    q.d.out = r.d_out;
    q.d.n_rows = st->n_streams;
    q.d.n_per = r.n_per_stream;
    q.d.pitch = r.n_per_stream;
    q.d.limit = (r.n_valid == 0 || r.n_valid > full) ? full : r.n_valid;
    q.d.pos = r.reseed ? initial_pos(st->gen) : st->pos;
    q.d.p = st->p;
    q.d.mode = r.f32 ? OUT_F32 : OUT_U32;
    q.seed = r.seed;
    q.gen = st->gen;
    q.reseed = r.reseed ? 1 : 0;
    g_new_pos[i] = advance_pos(st->gen, q.d.pos, r.n_per_stream);
    if (r.reseed)
      for (uint64_t r0 = 0; r0 < st->n_streams; r0 += 256)
        h_items[fill_at[FAM_SEED]++] =
            BatchItem{i, (uint32_t)std::min<uint64_t>(256, st->n_streams - r0), r0};
    if (r.n_per_stream > 0) {
      const int f = fill_family(r.st->gen, r.st->p, r.f32 != 0);
      const uint32_t per = rows_per_item(f, tile_of(f));
      for (uint64_t r0 = 0; r0 < st->n_streams; r0 += per)
        h_items[fill_at[f]++] =
            BatchItem{i, (uint32_t)std::min<uint64_t>(per, st->n_streams - r0), r0};
    }
  }
  for (int f = FAM_MLCG; f < FAM_COUNT; f++) {  // longest rows first within a family
    const bool per_row = kind_of(f) == FAM_MLCG || kind_of(f) == FAM_MT;
    std::sort(h_items + fam_off[f], h_items + fam_off[f] + fam_n[f],
              [&](const BatchItem& a, const BatchItem& c) {
                const uint64_t ca = h_reqs[a.req].d.n_per * (per_row ? a.rows : 1);
                const uint64_t cc = h_reqs[c.req].d.n_per * (per_row ? c.rows : 1);
                return ca > cc;
              });
  }

  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(d_reqs, h_reqs, n_reqs * sizeof(BatchReq), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      (total > 0 && cudaMemcpyAsync(d_items, h_items, total * sizeof(BatchItem),
                                    cudaMemcpyHostToDevice, s) != cudaSuccess) ||
      cudaMemsetAsync(d_counters, 0, kCounterBytes, s) != cudaSuccess) {
    cudaGetLastError();
    return PRNG_ECUDA;
  }
  auto queue = [&](int f) {
    return BatchQueue{d_reqs, d_items + fam_off[f], (uint32_t)fam_n[f], d_counters + f};
  };
  cudaError_t e = launch_batch_seed(queue(FAM_SEED), s);
  for (int f = FAM_MLCG; f < FAM_COUNT && e == cudaSuccess; f++) {
    if (fam_n[f] == 0) continue;
    const BatchQueue q = queue(f);
    const bool f32 = f >= FAM_KINDS;
    switch (kind_of(f)) {
      case FAM_MLCG: e = launch_batch_mlcg(q, tile_of(f), s); break;
      case FAM_XOR128: e = launch_batch_xor128(q, tile_of(f), f32, s); break;
      case FAM_RANMAR: e = launch_batch_ranmar(q, tile_of(f), f32, s); break;
      case FAM_MT: e = launch_batch_mt(q, tile_of(f), f32, s); break;
      default: e = launch_batch_ranlux(q, lux_p_of(f), tile_of(f), f32, s); break;
    }
  }
  if (e != cudaSuccess) return PRNG_ECUDA;
  for (uint32_t i = 0; i < n_reqs; i++) reqs[i].st->pos = g_new_pos[i];
  return PRNG_OK;
}
