// abi.cu -- the exported C ABI of libprng (declared in include/prng.h).
//
// Host side only: argument validation, device allocation of stream state,
// bookkeeping of the positions that are uniform over a handle's streams
// (RANLUX's place in its luxury block, MT19937's table index), and dispatch
// to the kernels.  Every draw is produced on the GPU.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/prng.h"
#include "common.cuh"
#include "handle.cuh"

using namespace prng;

namespace {

constexpr uint32_t kBlobMagic = 0x50524E47u;  // "PRNG"
constexpr uint32_t kBlobVersion = 1u;

// n_per outputs per stream in output mode `mode`; doubles take two draws
// each, so their fill runs the draw pipeline over 2 n_per draws.
int fill_impl(prng_state* st, void* d_out, uint64_t n_per, int mode, cudaStream_t s) {
  if (st == nullptr) return PRNG_ENULL;
  if (n_per == 0) return PRNG_OK;
  if (d_out == nullptr) return PRNG_ENULL;
  if ((reinterpret_cast<uintptr_t>(d_out) & (mode == OUT_F64 ? 7 : 3)) != 0) return PRNG_ESIZE;
  if (mode == OUT_F64) {
    if (n_per > UINT64_MAX / 2) return PRNG_ESIZE;
    // RANLUX's block position and MT19937's table index must be even so
    // that every pair sits inside the kernels' aligned units.
    if ((st->gen == RANLUX || st->gen == MT19937) && (st->pos & 1)) return PRNG_EPARITY;
    n_per *= 2;
  }
  if (st->n_streams > UINT64_MAX / n_per) return PRNG_ESIZE;
  FillDesc d{};
  d.state = st->d_state;
  d.n_rows = st->n_streams;
  d.n_per = n_per;
  d.out = d_out;
  d.pitch = n_per;
  d.limit = UINT64_MAX;
  d.pos = st->pos;
  d.p = st->p;
  d.mode = mode;
  d.jump = 0;
  const Tile t = default_tile(st->gen, st->p);
  cudaError_t e;
  switch (st->gen) {
    case RANMAR: e = launch_fill_ranmar(d, t, s); break;
    case RANLUX: e = launch_fill_ranlux(d, t, s); break;
    case MT19937: e = launch_fill_mt(d, t, s); break;
    default:  // GGL, XOR128, RANECU: lane-parallel tiles have 128 columns
      e = t.cols == 128 ? launch_fill_mlcg(st->gen, d, t, s) : launch_fill_simple(st->gen, d, t, s);
      break;
  }
  if (e != cudaSuccess) return PRNG_ECUDA;
  st->pos = advance_pos(st->gen, st->pos, n_per);
  return PRNG_OK;
}

// a^e mod m on the host, for a, m < 2^31 (products stay below 2^62).
uint64_t host_powmod(uint64_t a, uint64_t e, uint64_t m) {
  uint64_t r = 1, b = a % m;
  for (; e; e >>= 1) {
    if (e & 1) r = r * b % m;
    b = b * b % m;
  }
  return r;
}

int jump_impl(int gen, uint64_t x0, uint64_t first, uint64_t n, uint32_t n_chunks, void* d_out,
              int f32, cudaStream_t s) {
  if (gen < 0 || gen > 5) return PRNG_EGEN;
  if (gen != GGL && gen != RANECU && gen != XOR128 && gen != MT19937) return PRNG_EUNSUPPORTED;
  if (n == 0) return PRNG_OK;
  if (d_out == nullptr) return PRNG_ENULL;
  if (n_chunks == 0) return PRNG_ESIZE;
  if (n > ~0ull - first) return PRNG_ESIZE;
  if ((reinterpret_cast<uintptr_t>(d_out) & 3) != 0) return PRNG_ESIZE;
  if (gen == XOR128 || gen == MT19937) {
    if (gen == MT19937 && x0 > 0xFFFFFFFFull) return PRNG_ESEED;
    const cudaError_t e = gen == XOR128 ? launch_jump_xor128(x0, first, n, n_chunks, d_out, f32, s)
                                        : launch_jump_mt(x0, first, n, n_chunks, d_out,
                                                         f32 ? OUT_F32 : OUT_U32, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? PRNG_EALLOC : PRNG_ECUDA;
    }
    return PRNG_OK;
  }
  // The start moved `first` draws on: x_first = a^first x0 (per component).
  if (gen == GGL) {
    if (x0 == 0 || x0 >= 2147483647ull) return PRNG_ESEED;
    x0 = host_powmod(16807, first, 2147483647ull) * x0 % 2147483647ull;
  } else {
    uint64_t s1 = x0 & 0xFFFFFFFFull, s2 = x0 >> 32;
    if (s1 == 0 || s1 >= 2147483563ull || s2 == 0 || s2 >= 2147483399ull) return PRNG_ESEED;
    s1 = host_powmod(40014, first, 2147483563ull) * s1 % 2147483563ull;
    s2 = host_powmod(40692, first, 2147483399ull) * s2 % 2147483399ull;
    x0 = s1 | (s2 << 32);
  }
  // The generator's fill tile decides the kernel.  The lane-parallel one
  // runs a warp per chunk as asked; the staged one runs a thread per chunk,
  // so it cuts the sequence into more, shorter chunks when there are too
  // few to fill the GPU (the output is the same sequence).
  const Tile t = default_tile(gen, 0);
  const bool lanes = t.cols == 128;
  const uint64_t want = lanes ? n_chunks
                              : std::max<uint64_t>(n_chunks, std::min<uint64_t>((n + 255) / 256, 131072));
  const uint64_t L = (n + want - 1) / want;          // draws per chunk
  FillDesc d{};
  d.state = nullptr;
  d.n_rows = (n + L - 1) / L;                        // no empty chunk
  d.n_per = L;
  d.out = d_out;
  d.pitch = L;
  d.limit = n;
  d.x0 = x0;
  d.mode = f32 ? OUT_F32 : OUT_U32;
  d.jump = 1;
  const cudaError_t e = lanes ? launch_fill_mlcg(gen, d, t, s) : launch_fill_simple(gen, d, t, s);
  if (e != cudaSuccess) return PRNG_ECUDA;
  return PRNG_OK;
}

}  // namespace

namespace {

// Tiles compiled into the kernels, per generator family.
bool tile_supported(int gen, Tile t, int p = 0) {
  // RANLUX at p >= 97: also a 96-column staging tile (four delivered blocks
  // per flush), compiled for those levels only.
  if (gen == RANLUX && p >= 97 && t.threads == 64 && t.cols == 96 && t.stages == 1) return true;
  static const Tile simple[] = {{128, 32, 1}, {128, 32, 2}, {128, 64, 1}, {256, 32, 1}};
  static const Tile mlcg[] = {{128, 128, 1}, {256, 128, 1}};
  static const Tile lux[] = {{64, 48, 1}, {128, 48, 1}, {256, 48, 1},
                             {64, 56, 1}, {128, 56, 1}, {256, 56, 1}};   // 56: the per-row ring
  static const Tile mar[] = {{128, 128, 1}, {256, 128, 1}};
  static const Tile mt[] = {{64, 624, 1}, {128, 624, 1}, {256, 624, 1},
                            {32, 624, 2}, {64, 624, 2}, {128, 624, 2}, {256, 624, 2}};
  const Tile* list = simple;
  int n = 4;
  if ((gen == GGL || gen == RANECU) && t.cols == 128) { list = mlcg; n = 2; }
  else if (gen == RANLUX) { list = lux; n = 6; }
  else if (gen == RANMAR) { list = mar; n = 2; }
  else if (gen == MT19937) { list = mt; n = 7; }
  for (int i = 0; i < n; i++)
    if (list[i].threads == t.threads && list[i].cols == t.cols && list[i].stages == t.stages)
      return true;
  return false;
}

// Index of a RANLUX p: the standard levels 24, 48, 97, 223, 389, then the
// planar scheme's 120, 240, 408.
int lux_index(int p) {
  static const int P[8] = {24, 48, 97, 223, 389, 120, 240, 408};
  for (int i = 0; i < 8; i++)
    if (P[i] == p) return i;
  return 0;
}

// Per generator (RANLUX: per p) launch tiles; slot 5 + i is RANLUX p index i >= 1.
Tile g_tiles[13] = {{128, 128, 1}, {128, 32, 1}, {128, 128, 1}, {256, 128, 1}, {128, 48, 1},
                    {128, 624, 1}, {128, 48, 1}, {128, 48, 1}, {128, 48, 1}, {128, 48, 1},
                    {128, 48, 1}, {128, 48, 1}, {128, 48, 1}};

int tile_slot(int gen, int p) {
  if (gen != RANLUX) return gen;
  const int i = lux_index(p);
  return i == 0 ? RANLUX : 5 + i;
}

}  // namespace

namespace prng {

Tile default_tile(int gen, int p) { return g_tiles[tile_slot(gen, p)]; }

}  // namespace prng

extern "C" {

int prng_create(prng_state** out, prng_gen_t gen, uint64_t seed, uint32_t n_streams,
                uint32_t luxury) {
  if (out == nullptr) return PRNG_ENULL;
  *out = nullptr;
  const int g = (int)gen;
  if (g < 0 || g > 5) return PRNG_EGEN;
  int p = 0;
  if (g == RANLUX) {
    p = luxury_to_p(luxury);
    if (p < 0) return PRNG_ELUXURY;
  }
  if (n_streams == 0) return PRNG_ESIZE;
  prng_state* st = new (std::nothrow) prng_state;
  if (st == nullptr) return PRNG_EALLOC;
  st->gen = g;
  st->p = p;
  st->n_streams = n_streams;
  st->pos = initial_pos(g);
  st->d_state = nullptr;
  cudaGetDevice(&st->device);
  const size_t bytes = (size_t)n_streams * kWords[g] * sizeof(uint32_t);
  if (cudaMalloc(&st->d_state, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete st;
    return PRNG_EALLOC;
  }
  if (launch_seed(g, p, seed, n_streams, st->d_state, 0) != cudaSuccess ||
      cudaStreamSynchronize(0) != cudaSuccess) {
    cudaFree(st->d_state);
    delete st;
    return PRNG_ECUDA;
  }
  *out = st;
  return PRNG_OK;
}

int prng_reseed(prng_state* st, uint64_t seed, void* stream) {
  if (st == nullptr) return PRNG_ENULL;
  if (launch_seed(st->gen, st->p, seed, st->n_streams, st->d_state,
                  static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return PRNG_ECUDA;
  st->pos = initial_pos(st->gen);
  return PRNG_OK;
}

int prng_fill_u32(prng_state* st, uint32_t* d_out, uint64_t n_per_stream, void* stream) {
  return fill_impl(st, d_out, n_per_stream, OUT_U32, static_cast<cudaStream_t>(stream));
}

int prng_fill_f32(prng_state* st, float* d_out, uint64_t n_per_stream, void* stream) {
  return fill_impl(st, d_out, n_per_stream, OUT_F32, static_cast<cudaStream_t>(stream));
}

int prng_fill_f64(prng_state* st, double* d_out, uint64_t n_per_stream, void* stream) {
  return fill_impl(st, d_out, n_per_stream, OUT_F64, static_cast<cudaStream_t>(stream));
}

// The shift that leaves a draw's 24 top significant bits (reading R7): 31-bit
// GGL and RANECU words lose 7 bits, 32-bit XOR128 and MT19937 words 8, the
// 24-bit RANMAR and RANLUX words none.
static const uint32_t kFloatShift[6] = {7, 8, 7, 0, 0, 8};

int prng_float_shift(prng_gen_t gen, uint32_t* shift) {
  if (shift == nullptr) return PRNG_ENULL;
  if ((int)gen < 0 || (int)gen > 5) return PRNG_EGEN;
  *shift = kFloatShift[gen];
  return PRNG_OK;
}

int prng_ising_fused(prng_state* st, int8_t* d_spins, uint32_t L, uint32_t colour, uint32_t t4,
                     uint32_t t8, void* stream) {
  if (st == nullptr || d_spins == nullptr) return PRNG_ENULL;
  if (L < 2 || (L & 1) != 0 || L > 65534 || colour > 1) return PRNG_ESIZE;
  const uint64_t sites = (uint64_t)L * (L / 2);
  if (sites % st->n_streams != 0) return PRNG_ESIZE;
  FillDesc d{};
  d.state = st->d_state;
  d.n_rows = st->n_streams;
  d.n_per = sites / st->n_streams;
  d.out = d_spins;          // never written as words: the sink takes every draw
  d.pitch = d.n_per;
  d.limit = sites;
  d.pos = st->pos;
  d.p = st->p;
  d.mode = OUT_ISING;
  d.jump = 0;
  IsingSink& q = d.ising;
  q.spins = d_spins;
  q.L = L;
  q.half = L / 2;
  q.lg_half = 32;
  if ((q.half & (q.half - 1)) == 0)
    for (uint32_t b = 0; b < 32; b++)
      if ((1u << b) == q.half) q.lg_half = b;
  q.colour = colour;
  q.shift = kFloatShift[st->gen];
  q.t4 = t4;
  q.t8 = t8;
  q.vec4 = (L % 8 == 0 && (reinterpret_cast<uintptr_t>(d_spins) & 7) == 0) ? 1u : 0u;
  const Tile t = default_tile(st->gen, st->p);
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  switch (st->gen) {
    case RANMAR: e = launch_fill_ranmar(d, t, s); break;
    case RANLUX: e = launch_fill_ranlux(d, t, s); break;
    case MT19937: e = launch_fill_mt(d, t, s); break;
    default:
      e = t.cols == 128 ? launch_fill_mlcg(st->gen, d, t, s) : launch_fill_simple(st->gen, d, t, s);
      break;
  }
  if (e != cudaSuccess) return PRNG_ECUDA;
  st->pos = advance_pos(st->gen, st->pos, d.n_per);
  return PRNG_OK;
}

// XOR128 skips of at least this many steps use the GF(2) matrix power
// (about 128 column XORs per stream) instead of stepping.
constexpr uint64_t kXor128MatrixSkip = 256;
// MT19937 skips of at least this many outputs use the polynomial jump (about
// 19937 x 312 word XORs per stream) instead of stepping.
constexpr uint64_t kMtPolySkip = 1ull << 20;

int prng_skip(prng_state* st, uint64_t k, void* stream) {
  if (st == nullptr) return PRNG_ENULL;
  if (k == 0) return PRNG_OK;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (st->gen == GGL || st->gen == RANECU) {
    e = launch_skip_mlcg(st->gen, st->d_state, st->n_streams, k, s);
  } else if (st->gen == XOR128 && k >= kXor128MatrixSkip) {
    e = launch_skip_xor128(st->d_state, st->n_streams, k, s);
  } else if (st->gen == MT19937 && k >= kMtPolySkip) {
    // The tables move k words along the sequence; the read index stays.
    if (launch_skip_mt(st->d_state, st->n_streams, k, s) != cudaSuccess) return PRNG_ECUDA;
    return PRNG_OK;
  } else {
    FillDesc d{};
    d.state = st->d_state;
    d.n_rows = st->n_streams;
    d.n_per = k;
    d.out = nullptr;
    d.pitch = 0;
    d.limit = 0;
    d.pos = st->pos;
    d.p = st->p;
    const Tile t = default_tile(st->gen, st->p);
    switch (st->gen) {
      case RANMAR: e = launch_fill_ranmar(d, t, s); break;
      case RANLUX: e = launch_fill_ranlux(d, t, s); break;
      case MT19937: e = launch_fill_mt(d, t, s); break;
      default: e = launch_fill_simple(st->gen, d, t, s); break;
    }
  }
  if (e != cudaSuccess) return PRNG_ECUDA;
  st->pos = advance_pos(st->gen, st->pos, k);
  return PRNG_OK;
}

int prng_get_state(prng_state* st, void* h_buf, size_t* bytes) {
  if (st == nullptr || bytes == nullptr) return PRNG_ENULL;
  const uint64_t W = kWords[st->gen], n = st->n_streams;
  const size_t need = (8 + (size_t)n * W) * sizeof(uint32_t);
  if (h_buf == nullptr) {
    *bytes = need;
    return PRNG_OK;
  }
  if (*bytes < need) {
    *bytes = need;
    return PRNG_ESIZE;
  }
  std::vector<uint32_t> dev((size_t)n * W);
  if (cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpy(dev.data(), st->d_state, dev.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return PRNG_ECUDA;
  uint32_t* b = static_cast<uint32_t*>(h_buf);
  const uint32_t hdr[8] = {kBlobMagic, kBlobVersion, (uint32_t)st->gen, (uint32_t)st->p,
                           (uint32_t)n, (uint32_t)W, st->pos, 0u};
  std::memcpy(b, hdr, sizeof(hdr));
  uint32_t* body = b + 8;
  if (st->gen == MT19937) {
    std::memcpy(body, dev.data(), dev.size() * 4);
  } else {  // SoA on the device, stream-major in the blob
    for (uint64_t i = 0; i < n; i++)
      for (uint64_t w = 0; w < W; w++) body[i * W + w] = dev[w * n + i];
  }
  *bytes = need;
  return PRNG_OK;
}

int prng_set_state(prng_state* st, const void* h_buf, size_t bytes) {
  if (st == nullptr || h_buf == nullptr) return PRNG_ENULL;
  const uint64_t W = kWords[st->gen], n = st->n_streams;
  const size_t need = (8 + (size_t)n * W) * sizeof(uint32_t);
  if (bytes != need) return PRNG_EBLOB;
  const uint32_t* b = static_cast<const uint32_t*>(h_buf);
  if (b[0] != kBlobMagic || b[1] != kBlobVersion || b[2] != (uint32_t)st->gen ||
      b[3] != (uint32_t)st->p || b[4] != (uint32_t)n || b[5] != (uint32_t)W)
    return PRNG_EBLOB;
  const uint32_t pos = b[6];
  if ((st->gen == RANLUX && pos > 24) || (st->gen == MT19937 && pos > 624)) return PRNG_EBLOB;
  std::vector<uint32_t> dev((size_t)n * W);
  const uint32_t* body = b + 8;
  if (st->gen == MT19937) {
    std::memcpy(dev.data(), body, dev.size() * 4);
  } else {
    for (uint64_t i = 0; i < n; i++)
      for (uint64_t w = 0; w < W; w++) dev[w * n + i] = body[i * W + w];
  }
  if (cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpy(st->d_state, dev.data(), dev.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
    return PRNG_ECUDA;
  st->pos = pos;
  return PRNG_OK;
}

int prng_fill_jump_u32(prng_gen_t gen, uint64_t x0, uint64_t n, uint32_t n_chunks,
                       uint32_t* d_out, void* stream) {
  return jump_impl((int)gen, x0, 0, n, n_chunks, d_out, 0, static_cast<cudaStream_t>(stream));
}

int prng_fill_jump_f32(prng_gen_t gen, uint64_t x0, uint64_t n, uint32_t n_chunks,
                       float* d_out, void* stream) {
  return jump_impl((int)gen, x0, 0, n, n_chunks, d_out, 1, static_cast<cudaStream_t>(stream));
}

int prng_fill_jump_at_u32(prng_gen_t gen, uint64_t x0, uint64_t first, uint64_t n,
                          uint32_t n_chunks, uint32_t* d_out, void* stream) {
  return jump_impl((int)gen, x0, first, n, n_chunks, d_out, 0, static_cast<cudaStream_t>(stream));
}

int prng_fill_jump_at_f32(prng_gen_t gen, uint64_t x0, uint64_t first, uint64_t n,
                          uint32_t n_chunks, float* d_out, void* stream) {
  return jump_impl((int)gen, x0, first, n, n_chunks, d_out, 1, static_cast<cudaStream_t>(stream));
}

int prng_set_tile(prng_gen_t gen, uint32_t luxury, uint32_t threads, uint32_t cols,
                  uint32_t stages) {
  const int g = (int)gen;
  if (g < 0 || g > 5) return PRNG_EGEN;
  int p = 0;
  if (g == RANLUX) {
    p = luxury_to_p(luxury);
    if (p < 0) return PRNG_ELUXURY;
  }
  const Tile t{(int)threads, (int)cols, (int)stages};
  if (!tile_supported(g, t, p)) return PRNG_EUNSUPPORTED;
  g_tiles[tile_slot(g, p)] = t;
  return PRNG_OK;
}

int prng_get_tile(prng_gen_t gen, uint32_t luxury, uint32_t* threads, uint32_t* cols,
                  uint32_t* stages) {
  const int g = (int)gen;
  if (g < 0 || g > 5) return PRNG_EGEN;
  int p = 0;
  if (g == RANLUX) {
    p = luxury_to_p(luxury);
    if (p < 0) return PRNG_ELUXURY;
  }
  const Tile t = g_tiles[tile_slot(g, p)];
  if (threads) *threads = (uint32_t)t.threads;
  if (cols) *cols = (uint32_t)t.cols;
  if (stages) *stages = (uint32_t)t.stages;
  return PRNG_OK;
}

int prng_info(const prng_state* st, int32_t* gen, int32_t* p, uint32_t* n_streams,
              uint64_t* state_bytes) {
  if (st == nullptr) return PRNG_ENULL;
  if (gen) *gen = st->gen;
  if (p) *p = st->p;
  if (n_streams) *n_streams = (uint32_t)st->n_streams;
  if (state_bytes) *state_bytes = st->n_streams * (uint64_t)kWords[st->gen] * 4;
  return PRNG_OK;
}

int prng_host_alloc(void** h_out, size_t bytes) {
  if (h_out == nullptr) return PRNG_ENULL;
  if (bytes == 0) return PRNG_ESIZE;
  void* h = nullptr;
  if (cudaHostAlloc(&h, bytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
    cudaGetLastError();
    return PRNG_EALLOC;
  }
  void* d = nullptr;
  if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess || d != h) {
    cudaGetLastError();
    cudaFreeHost(h);
    return PRNG_ECUDA;
  }
  *h_out = h;
  return PRNG_OK;
}

int prng_host_free(void* h_buf) {
  if (h_buf == nullptr) return PRNG_OK;
  return cudaFreeHost(h_buf) == cudaSuccess ? PRNG_OK : PRNG_ECUDA;
}

void prng_destroy(prng_state* st) {
  if (st == nullptr) return;
  if (st->d_state) cudaFree(st->d_state);
  delete st;
}

const char* prng_strerror(int code) {
  switch (code) {
    case PRNG_OK: return "success";
    case PRNG_EGEN: return "unknown generator";
    case PRNG_ELUXURY: return "RANLUX luxury must be 0..4 or one of 24, 48, 97, 223, 389, 120, 240, 408";
    case PRNG_ESIZE: return "invalid size or alignment";
    case PRNG_ENULL: return "required pointer is NULL";
    case PRNG_EALLOC: return "device or host allocation failed";
    case PRNG_ECUDA: return "CUDA call or kernel launch failed";
    case PRNG_EUNSUPPORTED: return "operation not supported for this generator";
    case PRNG_EBLOB: return "state blob does not match this handle";
    case PRNG_ESEED: return "start value outside the generator's range";
    case PRNG_ESCRATCH: return "batch exceeds the fixed scratch of prng_batch_fill_noalloc";
    case PRNG_EPARITY: return "f64 fill of RANLUX or MT19937 at an odd draw position";
    default: return "unknown error code";
  }
}

}  // extern "C"
