// batcher.cu -- prng_batcher_*: a reusable batched-fill engine whose request
// set changes from launch to launch (the serving loop's per-tick pass).
//
// prng_batch_* plans one fixed request list and replays it as a graph.  A
// server instead forms a new set every tick from whatever has arrived, so
// the batcher owns a ring of NSLOT staging slots sized for a maximum number
// of requests and work items: each launch plans the new set into the next
// slot (pinned host buffers), copies it to the slot's device buffers, zeroes
// the slot's work counters and launches the family kernels on the caller's
// stream.  A slot is reused only after the launch that last used it has
// finished (its event), so the host can plan tick t+1 while tick t runs.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/prng.h"
#include "batch.cuh"
#include "handle.cuh"

using namespace prng;

namespace {

constexpr int kSlots = 4;

struct Slot {
  BatchReq* h_reqs = nullptr;     // pinned
  BatchItem* h_items = nullptr;   // pinned
  BatchReq* d_reqs = nullptr;
  BatchItem* d_items = nullptr;
  uint32_t* d_counters = nullptr;
  cudaEvent_t done = nullptr;
  bool pending = false;
};


}  // namespace

struct prng_batcher {
  uint32_t max_requests = 0;
  uint64_t max_items = 0;
  Slot slot[kSlots];
  int next = 0;
  std::vector<const prng_state*> handles;   // duplicate check, sized once
};

namespace {

void destroy_batcher(prng_batcher* b) {
  if (b == nullptr) return;
  for (auto& u : b->slot) {
    if (u.pending && u.done) cudaEventSynchronize(u.done);
    if (u.done) cudaEventDestroy(u.done);
    if (u.h_reqs) cudaFreeHost(u.h_reqs);
    if (u.h_items) cudaFreeHost(u.h_items);
    if (u.d_reqs) cudaFree(u.d_reqs);
    if (u.d_items) cudaFree(u.d_items);
    if (u.d_counters) cudaFree(u.d_counters);
  }
  delete b;
}

}  // namespace

extern "C" {

int prng_batcher_create(prng_batcher** out, uint32_t max_requests, uint64_t max_items) {
  if (out == nullptr) return PRNG_ENULL;
  *out = nullptr;
  if (max_requests == 0 || max_items == 0 || max_items > 0xFFFFFFFFull) return PRNG_ESIZE;
  prng_batcher* b = new (std::nothrow) prng_batcher;
  if (b == nullptr) return PRNG_EALLOC;
  b->max_requests = max_requests;
  b->max_items = max_items;
  try {
    b->handles.reserve(max_requests);
  } catch (...) {
    delete b;
    return PRNG_EALLOC;
  }
  for (auto& u : b->slot) {
    if (cudaMallocHost(&u.h_reqs, max_requests * sizeof(BatchReq)) != cudaSuccess ||
        cudaMallocHost(&u.h_items, max_items * sizeof(BatchItem)) != cudaSuccess ||
        cudaMalloc(&u.d_reqs, max_requests * sizeof(BatchReq)) != cudaSuccess ||
        cudaMalloc(&u.d_items, max_items * sizeof(BatchItem)) != cudaSuccess ||
        cudaMalloc(&u.d_counters, FAM_COUNT * sizeof(uint32_t)) != cudaSuccess) {
      cudaGetLastError();
      destroy_batcher(b);
      return PRNG_EALLOC;
    }
    if (cudaEventCreateWithFlags(&u.done, cudaEventDisableTiming) != cudaSuccess) {
      destroy_batcher(b);
      return PRNG_ECUDA;
    }
  }
  *out = b;
  return PRNG_OK;
}

int prng_batcher_launch(prng_batcher* b, const prng_fill_req* reqs, uint32_t n_reqs, void* stream) {
  if (b == nullptr) return PRNG_ENULL;
  if (n_reqs == 0) return PRNG_OK;
  if (reqs == nullptr) return PRNG_ENULL;
  if (n_reqs > b->max_requests) return PRNG_ESIZE;
  uint64_t fam_n[FAM_COUNT] = {};
  for (uint32_t i = 0; i < n_reqs; i++) {
    const prng_fill_req& r = reqs[i];
    if (r.st == nullptr) return PRNG_ENULL;
    if (r.n_per_stream > 0 && r.d_out == nullptr) return PRNG_ENULL;
    if ((reinterpret_cast<uintptr_t>(r.d_out) & 3) != 0) return PRNG_ESIZE;
    if (r.n_per_stream > 0 && r.st->n_streams > UINT64_MAX / r.n_per_stream) return PRNG_ESIZE;
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
    fam_off[f] = (uint32_t)std::min<uint64_t>(total, b->max_items);
    total += fam_n[f];
  }
  if (total > b->max_items) return PRNG_ESIZE;
  // A handle may appear once per launch (its streams advance once): sorted
  // copy of the handles, adjacent equal ones rejected.
  b->handles.clear();
  for (uint32_t i = 0; i < n_reqs; i++) b->handles.push_back(reqs[i].st);
  std::sort(b->handles.begin(), b->handles.end());
  if (std::adjacent_find(b->handles.begin(), b->handles.end()) != b->handles.end()) return PRNG_EBLOB;

  Slot& u = b->slot[b->next];
  if (u.pending) {
    if (cudaEventSynchronize(u.done) != cudaSuccess) return PRNG_ECUDA;
    u.pending = false;
  }
  uint32_t at[FAM_COUNT];
  std::memcpy(at, fam_off, sizeof(at));
  for (uint32_t i = 0; i < n_reqs; i++) {
    const prng_fill_req& r = reqs[i];
    prng_state* st = r.st;
    BatchReq& q = u.h_reqs[i];
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
    st->pos = advance_pos(st->gen, q.d.pos, r.n_per_stream);
    if (r.reseed)
      for (uint64_t r0 = 0; r0 < st->n_streams; r0 += 256)
        u.h_items[at[FAM_SEED]++] =
            BatchItem{i, (uint32_t)std::min<uint64_t>(256, st->n_streams - r0), r0};
    if (r.n_per_stream > 0) {
      const int f = fill_family(r.st->gen, r.st->p, r.f32 != 0);
      const uint32_t per = rows_per_item(f, tile_of(f));
      for (uint64_t r0 = 0; r0 < st->n_streams; r0 += per)
        u.h_items[at[f]++] = BatchItem{i, (uint32_t)std::min<uint64_t>(per, st->n_streams - r0), r0};
    }
  }
  for (int f = FAM_MLCG; f < FAM_COUNT; f++) {  // longest rows first within a family
    const bool per_row = kind_of(f) == FAM_MLCG || kind_of(f) == FAM_MT;
    std::sort(u.h_items + fam_off[f], u.h_items + fam_off[f] + fam_n[f],
              [&](const BatchItem& a, const BatchItem& c) {
                const uint64_t ca = u.h_reqs[a.req].d.n_per * (per_row ? a.rows : 1);
                const uint64_t cc = u.h_reqs[c.req].d.n_per * (per_row ? c.rows : 1);
                return ca > cc;
              });
  }
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(u.d_reqs, u.h_reqs, n_reqs * sizeof(BatchReq), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      (total > 0 && cudaMemcpyAsync(u.d_items, u.h_items, total * sizeof(BatchItem),
                                    cudaMemcpyHostToDevice, s) != cudaSuccess) ||
      cudaMemsetAsync(u.d_counters, 0, FAM_COUNT * sizeof(uint32_t), s) != cudaSuccess) {
    cudaGetLastError();
    return PRNG_ECUDA;
  }
  auto queue = [&](int f) {
    return BatchQueue{u.d_reqs, u.d_items + fam_off[f], (uint32_t)fam_n[f], u.d_counters + f};
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
  if (e != cudaSuccess || cudaEventRecord(u.done, s) != cudaSuccess) return PRNG_ECUDA;
  u.pending = true;
  b->next = (b->next + 1) % kSlots;
  return PRNG_OK;
}

void prng_batcher_destroy(prng_batcher* b) { destroy_batcher(b); }

}  // extern "C"
