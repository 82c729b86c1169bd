// batch_host.cu -- planning and launching of batched fills (prng_batch_*).
//
// A plan turns a list of fill requests on distinct handles into work items
// per generator family (a range of one request's streams each, longest
// first) and keeps them on the device.  A launch writes the per-request
// descriptors (start positions, re-seed flags) into one of two pinned
// buffers, and replays a CUDA graph that copies them to the device, zeroes
// the work counters, runs the re-seeding pass and then the persistent
// family kernels on forked branches, so a family's tail overlaps the next
// family's start.  The two descriptor buffers, each with its own graph,
// let the host prepare launch k+1 while launch k runs.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/prng.h"
#include "batch.cuh"
#include "handle.cuh"

using namespace prng;

namespace {

struct Buffers {
  BatchReq* h_reqs = nullptr;     // pinned
  BatchReq* d_reqs = nullptr;
  uint32_t* d_counters = nullptr; // FAM_COUNT counters
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t done = nullptr;     // recorded after the graph launch that used this buffer
  bool pending = false;
};

}  // namespace

struct prng_batch {
  std::vector<prng_fill_req> reqs;
  BatchItem* d_items = nullptr;
  uint32_t fam_off[FAM_COUNT] = {};
  uint32_t fam_n[FAM_COUNT] = {};
  Tile fam_tile[FAM_COUNT] = {};
  Buffers buf[2];
  int next = 0;
  cudaStream_t cap = nullptr;
  cudaStream_t branch[FAM_COUNT] = {};
  cudaEvent_t fork = nullptr, join[FAM_COUNT] = {};
  int device = 0;
};

namespace {

void destroy_batch(prng_batch* b) {
  if (b == nullptr) return;
  for (auto& u : b->buf) {
    if (u.pending && u.done) cudaEventSynchronize(u.done);
    if (u.exec) cudaGraphExecDestroy(u.exec);
    if (u.done) cudaEventDestroy(u.done);
    if (u.h_reqs) cudaFreeHost(u.h_reqs);
    if (u.d_reqs) cudaFree(u.d_reqs);
    if (u.d_counters) cudaFree(u.d_counters);
  }
  if (b->d_items) cudaFree(b->d_items);
  for (int f = 0; f < FAM_COUNT; f++) {
    if (b->branch[f]) cudaStreamDestroy(b->branch[f]);
    if (b->join[f]) cudaEventDestroy(b->join[f]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

// Record the pass for buffer u as a graph on the capture stream.
cudaError_t capture(prng_batch* b, Buffers& u) {
  const size_t nreq = b->reqs.size();
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaMemcpyAsync(u.d_reqs, u.h_reqs, nreq * sizeof(BatchReq), cudaMemcpyHostToDevice, b->cap);
  cudaMemsetAsync(u.d_counters, 0, FAM_COUNT * sizeof(uint32_t), b->cap);
  auto queue = [&](int f) {
    return BatchQueue{u.d_reqs, b->d_items + b->fam_off[f], b->fam_n[f], u.d_counters + f};
  };
  launch_batch_seed(queue(FAM_SEED), b->cap);
  cudaEventRecord(b->fork, b->cap);
  int used[FAM_COUNT];
  int nused = 0;
  for (int f = FAM_MLCG; f < FAM_COUNT; f++) {
    if (b->fam_n[f] == 0) continue;
    cudaStream_t s = b->branch[f];
    cudaStreamWaitEvent(s, b->fork, 0);
    const BatchQueue q = queue(f);
    const Tile t = b->fam_tile[f];
    const bool f32 = is_f32_family(f);
    switch (kind_of(f)) {
      case FAM_MLCG: launch_batch_mlcg(q, t, s); break;
      case FAM_XOR128: launch_batch_xor128(q, t, f32, s); break;
      case FAM_RANMAR: launch_batch_ranmar(q, t, f32, s); break;
      case FAM_MT: launch_batch_mt(q, t, f32, s); break;
      default: launch_batch_ranlux(q, lux_p_of(f), t, f32, s); break;
    }
    cudaEventRecord(b->join[f], s);
    used[nused++] = f;
  }
  for (int i = 0; i < nused; i++) cudaStreamWaitEvent(b->cap, b->join[used[i]], 0);
  const cudaError_t le = cudaGetLastError();
  e = cudaStreamEndCapture(b->cap, &g);
  if (le != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return le;
  }
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(&u.exec, g, 0);
  cudaGraphDestroy(g);
  return e;
}

}  // namespace

extern "C" {

int prng_batch_create(prng_batch** out, const prng_fill_req* reqs, uint32_t n_reqs) {
  if (out == nullptr) return PRNG_ENULL;
  *out = nullptr;
  if (n_reqs == 0) return PRNG_ESIZE;
  if (reqs == nullptr) return PRNG_ENULL;
  std::vector<const prng_state*> seen;
  seen.reserve(n_reqs);
  for (uint32_t i = 0; i < n_reqs; i++) {
    const prng_fill_req& r = reqs[i];
    if (r.st == nullptr) return PRNG_ENULL;
    if (r.n_per_stream > 0 && r.d_out == nullptr) return PRNG_ENULL;
    if ((reinterpret_cast<uintptr_t>(r.d_out) & 3) != 0) return PRNG_ESIZE;
    if (r.n_per_stream > 0 && r.st->n_streams > UINT64_MAX / r.n_per_stream) return PRNG_ESIZE;
    seen.push_back(r.st);
  }
  std::sort(seen.begin(), seen.end());
  if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) return PRNG_EBLOB;

  prng_batch* b = new (std::nothrow) prng_batch;
  if (b == nullptr) return PRNG_EALLOC;
  b->reqs.assign(reqs, reqs + n_reqs);
  cudaGetDevice(&b->device);

  // Work items per family, longest rows first.
  std::vector<std::vector<BatchItem>> items(FAM_COUNT);
  std::vector<std::vector<uint64_t>> cost(FAM_COUNT);
  for (int f = 0; f < FAM_COUNT; f++) {
    b->fam_tile[f] = tile_of(f);
  }
  for (uint32_t i = 0; i < n_reqs; i++) {
    const prng_fill_req& r = reqs[i];
    const prng_state* st = r.st;
    if (r.reseed) {
      for (uint64_t r0 = 0; r0 < st->n_streams; r0 += 256) {
        const uint32_t rows = (uint32_t)std::min<uint64_t>(256, st->n_streams - r0);
        items[FAM_SEED].push_back(BatchItem{i, rows, r0});
        cost[FAM_SEED].push_back(0);
      }
    }
    if (r.n_per_stream == 0) continue;
    const int kind = family_of(st->gen, st->p);
    const int f = (r.f32 && kind != FAM_MLCG) ? kind + FAM_F32 : kind;  // MLCG mixes dtypes
    const uint32_t per = rows_per_item(f, b->fam_tile[f]);
    for (uint64_t r0 = 0; r0 < st->n_streams; r0 += per) {
      const uint32_t rows = (uint32_t)std::min<uint64_t>(per, st->n_streams - r0);
      items[f].push_back(BatchItem{i, rows, r0});
      cost[f].push_back(r.n_per_stream * (kind == FAM_MLCG || kind == FAM_MT ? rows : 1));
    }
  }
  std::vector<BatchItem> all;
  for (int f = 0; f < FAM_COUNT; f++) {
    std::vector<size_t> order(items[f].size());
    for (size_t k = 0; k < order.size(); k++) order[k] = k;
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t a, size_t c) { return cost[f][a] > cost[f][c]; });
    b->fam_off[f] = (uint32_t)all.size();
    b->fam_n[f] = (uint32_t)order.size();
    for (size_t k : order) all.push_back(items[f][k]);
  }

  int rc = PRNG_OK;
  if (cudaMalloc(&b->d_items, std::max<size_t>(1, all.size()) * sizeof(BatchItem)) != cudaSuccess)
    rc = PRNG_EALLOC;
  if (rc == PRNG_OK && !all.empty() &&
      cudaMemcpy(b->d_items, all.data(), all.size() * sizeof(BatchItem), cudaMemcpyHostToDevice) !=
          cudaSuccess)
    rc = PRNG_ECUDA;
  for (auto& u : b->buf) {
    if (rc != PRNG_OK) break;
    if (cudaMallocHost(&u.h_reqs, n_reqs * sizeof(BatchReq)) != cudaSuccess ||
        cudaMalloc(&u.d_reqs, n_reqs * sizeof(BatchReq)) != cudaSuccess ||
        cudaMalloc(&u.d_counters, FAM_COUNT * sizeof(uint32_t)) != cudaSuccess)
      rc = PRNG_EALLOC;
    else if (cudaEventCreateWithFlags(&u.done, cudaEventDisableTiming) != cudaSuccess)
      rc = PRNG_ECUDA;
  }
  if (rc == PRNG_OK) {
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
      rc = PRNG_ECUDA;
    for (int f = 0; f < FAM_COUNT && rc == PRNG_OK; f++)
      if (cudaStreamCreateWithFlags(&b->branch[f], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&b->join[f], cudaEventDisableTiming) != cudaSuccess)
        rc = PRNG_ECUDA;
  }
  if (rc != PRNG_OK) {
    cudaGetLastError();
    destroy_batch(b);
    return rc;
  }
  *out = b;
  return PRNG_OK;
}

int prng_batch_launch(prng_batch* b, void* stream) {
  if (b == nullptr) return PRNG_ENULL;
  Buffers& u = b->buf[b->next];
  if (u.pending) {  // the pinned buffer may still be in flight from two launches ago
    if (cudaEventSynchronize(u.done) != cudaSuccess) return PRNG_ECUDA;
    u.pending = false;
  }
  for (size_t i = 0; i < b->reqs.size(); i++) {
    const prng_fill_req& r = b->reqs[i];
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
    q.d.jump = 0;
    q.seed = r.seed;
    q.gen = st->gen;
    q.reseed = r.reseed ? 1 : 0;
    st->pos = advance_pos(st->gen, q.d.pos, r.n_per_stream);
  }
  if (u.exec == nullptr) {
    const cudaError_t e = capture(b, u);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return PRNG_ECUDA;
    }
  }
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaGraphLaunch(u.exec, s) != cudaSuccess || cudaEventRecord(u.done, s) != cudaSuccess)
    return PRNG_ECUDA;
  u.pending = true;
  b->next ^= 1;
  return PRNG_OK;
}

int prng_batch_info(const prng_batch* b, uint32_t* n_requests, uint64_t* n_items,
                    uint64_t* n_numbers) {
  if (b == nullptr) return PRNG_ENULL;
  uint64_t items = 0, numbers = 0;
  for (int f = 0; f < FAM_COUNT; f++) items += b->fam_n[f];
  for (const auto& r : b->reqs) {
    const uint64_t full = r.st->n_streams * r.n_per_stream;
    numbers += (r.n_valid == 0 || r.n_valid > full) ? full : r.n_valid;
  }
  if (n_requests) *n_requests = (uint32_t)b->reqs.size();
  if (n_items) *n_items = items;
  if (n_numbers) *n_numbers = numbers;
  return PRNG_OK;
}

void prng_batch_destroy(prng_batch* b) { destroy_batch(b); }

}  // extern "C"
