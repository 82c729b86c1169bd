/*
 * prng.h -- C ABI of libprng, a GB300 (sm_103a) library for bulk uniform
 * pseudo-random numbers from the six generators of V. Demchik,
 * "Pseudo-random number generators for Monte Carlo simulations on GPUs"
 * (arXiv:1003.1898): GGL (Section 3.2), XOR128 (Section 3.3), RANECU
 * (Section 3.4), RANMAR (Section 3.5), RANLUX (Section 3.6) and MT19937
 * (Section 3.7), with the recurrences of Appendix A.
 *
 * Conventions shared by every entry point
 *   - Return value: 0 on success, a negative PRNG_E* code otherwise
 *     (prng_strerror() names it).  Arguments are validated on the host
 *     before anything is launched; a rejected call changes nothing.
 *   - Pointers named d_* are CUDA device pointers owned by the caller; the
 *     library never frees them.  Host pointers are named h_*.  An output
 *     d_* may also be host memory from prng_host_alloc (written over the
 *     host link).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Fills are asynchronous on that stream; the caller orders
 *     work on one handle (a handle is not thread-safe).
 *   - Outputs are stream-major: element (i, j) of a fill, the j-th new draw
 *     of stream i, is at d_out[i * n_per_stream + j].
 *   - u32 outputs: GGL x_n in [1, 2^31-2]; XOR128 the new word; RANECU the
 *     combined value in [1, 2147483562]; RANMAR and RANLUX the 24-bit
 *     integer (the paper's float value times 2^24); MT19937 the tempered
 *     word.  f32 outputs are the exact scaling (v >> sh) * 2^-24 in [0, 1),
 *     sh = 7 (GGL, RANECU), 8 (XOR128, MT19937), 0 (RANMAR, RANLUX).
 */
#ifndef PRNG_H
#define PRNG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum prng_gen {
  PRNG_GGL = 0,      /* x <- 16807 x mod (2^31 - 1)                       (Section 3.2) */
  PRNG_XOR128 = 1,   /* Marsaglia xorshift, shifts 11/19/8                 (Section 3.3) */
  PRNG_RANECU = 2,   /* L'Ecuyer combination of two MLCGs                  (Section 3.4) */
  PRNG_RANMAR = 3,   /* LFG(97,33,-) mod 2^24 combined with a Weyl sequence (Section 3.5) */
  PRNG_RANLUX = 4,   /* RCARRY SWB(2^24,10,24) with luxury decimation      (Section 3.6) */
  PRNG_MT19937 = 5   /* Mersenne twister                                   (Section 3.7) */
} prng_gen_t;

enum {
  PRNG_OK = 0,
  PRNG_EGEN = -1,        /* unknown generator                                   */
  PRNG_ELUXURY = -2,     /* RANLUX luxury not in {0..4, 24, 48, 97, 223, 389, 120, 240, 408} */
  PRNG_ESIZE = -3,       /* zero streams/chunks, or a size that overflows        */
  PRNG_ENULL = -4,       /* a required pointer is NULL                           */
  PRNG_EALLOC = -5,      /* device allocation failed                             */
  PRNG_ECUDA = -6,       /* a CUDA call or launch failed                         */
  PRNG_EUNSUPPORTED = -7,/* operation not defined for this generator             */
  PRNG_EBLOB = -8,       /* malformed or mismatched state blob                   */
  PRNG_ESEED = -9,       /* jump start value outside the generator's range       */
  PRNG_ESCRATCH = -10,   /* batch larger than prng_batch_fill_noalloc's fixed scratch */
  PRNG_EPARITY = -11     /* f64 fill of RANLUX/MT19937 at an odd block position */
};

/* Opaque handle: one generator type, n_streams independent streams, their
 * state resident in device memory owned by the handle. */
typedef struct prng_state prng_state;

/* Create a handle with n_streams streams of generator `gen` on the current
 * CUDA device and seed them on the device (one launch, then a synchronise).
 * Stream i is seeded from s = splitmix64(seed + i) (SplitMix64 of Steele,
 * Lea and Flood: add 0x9E3779B97F4A7C15, then its mix64 finaliser), mapped
 * into the generator's seed range:
 *   GGL x0 = 1 + s mod (2^31-2); XOR128 (x,y,z,w) = the 32-bit halves of s and
 *   of splitmix64(s) (w = 1 if all are 0); RANECU s1 = 1 + lo32(s) mod
 *   (m1-1), s2 = 1 + hi32(s) mod (m2-1); RANMAR RMARIN(ij = lo32(s) mod
 *   31329, kl = hi32(s) mod 30082) (Section 3.5); RANLUX table from the MLCG
 *   40014 mod 2147483563 started at s mod 2147483563 (19780503 if 0);
 *   MT19937 init_genrand(lo32(s)).
 * `luxury` selects RANLUX's p: levels 0..4 or p in {24,48,97,223,389}
 * (Appendix A "RANLUX"), or p in {120,240,408}, the planar scheme of
 * Section 3.6 (24 numbers delivered, then 96, 216 or 384 discarded; its
 * first level is p = 48).  It is ignored for the other generators.
 * On success *out owns device memory until prng_destroy(). */
int prng_create(prng_state **out, prng_gen_t gen, uint64_t seed, uint32_t n_streams,
                uint32_t luxury);

/* Re-seed every stream of an existing handle in place, as prng_create would
 * with `seed`; asynchronous on `stream`, allocates nothing. */
int prng_reseed(prng_state *st, uint64_t seed, void *stream);

/* Write the next n_per_stream draws of every stream to d_out (stream-major,
 * n_streams * n_per_stream elements) and advance every stream by
 * n_per_stream.  n_per_stream = 0 is a no-op.  d_out needs 4-byte alignment;
 * 16-byte alignment with n_per_stream % 4 == 0 takes the vector-store path. */
int prng_fill_u32(prng_state *st, uint32_t *d_out, uint64_t n_per_stream, void *stream);
int prng_fill_f32(prng_state *st, float *d_out, uint64_t n_per_stream, void *stream);

/* Doubles from pairs of draws (Sections 3.1 and 4 ask for doubles built
 * from several draws rather than a widened single one): element (i, j) of
 * d_out (stream-major, n_streams * n_per_stream doubles) is made of draws
 * 2j+1 (high part) and 2j+2 (low part) of stream i counted from this call,
 * and every stream advances by 2 n_per_stream draws.  24-bit generators
 * (RANMAR, RANLUX) give (a 2^24 + b) 2^-48; the others give the top 27
 * bits of a over the top 26 bits of b, 2^-53 (31-bit words: (a >> 4) 2^26 +
 * (b >> 5); 32-bit words: (a >> 5) 2^26 + (b >> 6)).  Every value is exact
 * and in [0, 1).  d_out needs 8-byte alignment.  RANLUX and MT19937 need an
 * even number of draws taken since seeding (their position inside the
 * 24-draw block or the 624-word table must be even): PRNG_EPARITY
 * otherwise, with nothing written. */
int prng_fill_f64(prng_state *st, double *d_out, uint64_t n_per_stream, void *stream);

/* Advance every stream by k draws without writing them (same result as a
 * fill of k whose output is thrown away).  GGL and RANECU jump in O(log k)
 * by a^k mod m (Appendix A, eq. MLCG); XOR128 (k >= 256) by T^k, the k-th
 * power of its 128 x 128 step matrix over GF(2) (Appendix A, "XORShift",
 * matrix form), formed on the host in O(log k); MT19937 (k >= 2^20) by the
 * jump polynomial t^(k-1) mod phi (phi the degree-19937 characteristic
 * polynomial of one word step, Section 3.7) and one more step, each table
 * moving k words along its word sequence (about 6 million word XORs per
 * stream, whatever k; the read index is unchanged, so a later state blob
 * differs from a stepped one's in layout, not in the draws); the others
 * step. */
int prng_skip(prng_state *st, uint64_t k, void *stream);

/* Checkpoint.  prng_get_state copies the handle's full state into h_buf
 * (host memory, *bytes long); with h_buf == NULL it only stores the size
 * needed in *bytes.  It synchronises the device.  prng_set_state restores
 * a blob taken from a handle of the same generator, luxury and n_streams
 * (PRNG_EBLOB otherwise).  Blob layout: 8 uint32 header words {magic
 * 0x50524E47, version 1, gen, p, n_streams, words_per_stream, position,
 * 0} followed by n_streams * words_per_stream uint32 words, stream-major. */
int prng_get_state(prng_state *st, void *h_buf, size_t *bytes);
int prng_set_state(prng_state *st, const void *h_buf, size_t bytes);

/* Single-sequence jump-ahead fill (GGL, RANECU, XOR128 and MT19937): write draws
 * 1..n of the one sequence started at x0 to d_out[0..n), computed as
 * n_chunks contiguous chunks in parallel, L = ceil(n / n_chunks) draws each
 * (GGL and RANECU on their thread-per-stream tile, and XOR128, cut the
 * sequence into more, shorter chunks when n_chunks is too few to fill the
 * GPU; the output is the same).
 * GGL: x0 in [1, 2^31-2], chunk c starts from a^(c*L) x0 mod m by
 * square-and-multiply (Appendix A, eq. MLCG).  RANECU: x0 = s1 | (s2 << 32)
 * with s1 in [1, m1-1], s2 in [1, m2-1], both components jumped separately.
 * XOR128: any x0; the sequence starts from the state the stream seeding map
 * gives for the per-stream value s = x0 ((x, y) = halves of x0, (z, w) =
 * halves of splitmix64(x0)), and chunk c starts from T^(c*L) of it over
 * GF(2) (Appendix A, "XORShift", matrix form).  The XOR128 form may cut the
 * sequence into more, shorter chunks than asked (at least 131072 when n
 * allows 64 draws each; the output is the same), and takes a
 * stream-ordered scratch array of 16 bytes per chunk (PRNG_EALLOC if that
 * fails).  MT19937: x0 < 2^32, the sequence of init_genrand(x0); chunk c
 * starts from its table moved c*L words on, built in log2(n_chunks)
 * doubling passes of the jump polynomial (about 6 million word XORs per
 * chunk, so a few thousand chunks is the useful range), with a scratch
 * array of 2.5 KB per chunk.  The MT19937 form merges the chunks into fewer,
 * longer ones when more are asked than one wave of warps holds (27 per SM,
 * a warp per chunk; the output is the same).  The scratch arrays come from a stream-ordered
 * memory pool that the library creates on first use on each device and
 * that keeps its memory until the process exits, so repeated jump fills do
 * not allocate afresh.  Other generators return PRNG_EUNSUPPORTED. */
int prng_fill_jump_u32(prng_gen_t gen, uint64_t x0, uint64_t n, uint32_t n_chunks,
                       uint32_t *d_out, void *stream);
int prng_fill_jump_f32(prng_gen_t gen, uint64_t x0, uint64_t n, uint32_t n_chunks,
                       float *d_out, void *stream);

/* The same single-sequence fill from position `first` on: draws first+1 ..
 * first+n of the sequence started at x0 go to d_out[0..n), so that disjoint
 * ranges (one per GPU, say) tile one long sequence.  The start is moved
 * `first` draws on once (GGL, RANECU: a^first by square-and-multiply on the
 * host; XOR128: T^first over GF(2); MT19937: one application of the jump
 * polynomial of `first`), then chunked as above.  PRNG_ESIZE if first + n
 * overflows 64 bits; otherwise as prng_fill_jump_*; first = 0 is exactly
 * prng_fill_jump_*. */
int prng_fill_jump_at_u32(prng_gen_t gen, uint64_t x0, uint64_t first, uint64_t n,
                          uint32_t n_chunks, uint32_t *d_out, void *stream);
int prng_fill_jump_at_f32(prng_gen_t gen, uint64_t x0, uint64_t first, uint64_t n,
                          uint32_t n_chunks, float *d_out, void *stream);

/* ---------------------------------------------------------------- batches
 * Many fills on distinct handles run as one pass: the plan cuts every
 * request into work items (a range of its streams), orders each generator
 * family's items longest first and keeps them on the device; a launch runs
 * the optional re-seeding of the flagged handles and then one persistent
 * kernel per generator family that pops items from a device counter, as one
 * CUDA graph launch.  The draws are exactly those of prng_reseed followed by
 * prng_fill_u32/f32 on each handle alone (the paper's generators, Sections
 * 3.2-3.7, unchanged). */
typedef struct prng_fill_req {
  prng_state *st;         /* handle to fill; each handle at most once per batch */
  void *d_out;            /* device output, stream-major, pitch n_per_stream   */
  uint64_t n_per_stream;  /* draws per stream (the handle advances by this)   */
  uint64_t n_valid;       /* elements written: the first n_valid of the block
                             (0 = all n_streams * n_per_stream)               */
  uint64_t seed;          /* base seed used when reseed is set                */
  uint32_t f32;           /* 0: uint32 output, 1: float output                */
  uint32_t reseed;        /* 1: re-seed the handle from `seed` first          */
} prng_fill_req;

typedef struct prng_batch prng_batch;

/* Plan a batch.  Copies the request list (handles must stay alive and must
 * not be destroyed before the batch); allocates the work items, two
 * descriptor buffers and the work counters.  PRNG_EBLOB if a handle appears
 * twice. */
int prng_batch_create(prng_batch **out, const prng_fill_req *reqs, uint32_t n_reqs);

/* Run the batch once on `stream` (asynchronous).  Every handle's position
 * advances as after its own fill.  The first launch on each of the two
 * descriptor buffers captures the CUDA graph that later launches replay;
 * launch k+2 waits on the host for launch k to finish with its buffer.
 * Launches of one batch must be issued to one stream. */
int prng_batch_launch(prng_batch *b, void *stream);

/* Requests, work items and numbers written per launch. */
int prng_batch_info(const prng_batch *b, uint32_t *n_requests, uint64_t *n_items,
                    uint64_t *n_numbers);

/* Wait for the batch's launches and free it (NULL accepted). */
void prng_batch_destroy(prng_batch *b);

/* A batched-fill engine for request sets that change from launch to launch
 * (a serving loop's ticks).  It owns a ring of staging slots, each sized for
 * max_requests requests and max_items work items (work items as for
 * prng_batch_create).  prng_batcher_launch plans the given requests into
 * the next slot, copies them to the device and launches the same family
 * kernels as a batch, on `stream`, asynchronously; a slot is reused once the
 * launch that last used it has completed (the call waits for that on the
 * host).  Each handle at most once per launch; handles advance as after
 * their own fills.  PRNG_ESIZE when a launch exceeds the slot size. */
typedef struct prng_batcher prng_batcher;
int prng_batcher_create(prng_batcher **out, uint32_t max_requests, uint64_t max_items);
int prng_batcher_launch(prng_batcher *b, const prng_fill_req *reqs, uint32_t n_reqs, void *stream);
void prng_batcher_destroy(prng_batcher *b);

/* ---------------------------------------------------------------- Ising
 * Checkerboard Metropolis half-sweeps of periodic 2-D Ising lattices (J = 1,
 * h = 0) that consume the generators' draws -- the Monte Carlo use the
 * paper's generators are built for (Section 3.5 cites RANMAR's Ising
 * simulations).  Spins are +1/-1 in int8, row-major L x L, L even.  Only
 * sites of colour `colour` ((x + y) % 2) are visited; the site of colour
 * rank k (k = y L/2 + x/2) uses d_draws[k], whose 24-bit value
 * r = d_draws[k] >> shift (shift = the generator's float shift: 7 for GGL
 * and RANECU, 8 for XOR128 and MT19937, 0 for RANMAR and RANLUX) accepts
 * the flip when dE = 2 s (sum of the four neighbours) <= 0, or when r < t4
 * (dE = 4) or r < t8 (dE = 8).  d_draws is typically a handle's u32 fill of
 * L*L/2 draws (stream-major). */
typedef struct prng_ising_req {
  int8_t *d_spins;
  const uint32_t *d_draws;
  uint32_t L;
  uint32_t colour;
  uint32_t shift;
  uint32_t t4;
  uint32_t t8;
  /* Layout of the draws: pitch = 0 means site k takes d_draws[k] (one
   * stream-major block).  Otherwise site k takes d_draws[(k / per) * pitch
   * + k % per]: the half-sweep's block of per draws per stream sits inside
   * rows of `pitch` words, so one fill of several half-sweeps' draws serves
   * them all (d_draws pointing at the half-sweep's column offset). */
  uint32_t per;
  uint32_t pitch;
} prng_ising_req;

/* One half-sweep of each of the n lattices, asynchronously on `stream`.
 * The descriptors are passed by value to the kernels (no allocation).
 * Lattices with L a multiple of 16, d_spins and d_draws 16-byte aligned and
 * (pitch = 0 or per a multiple of 8 and pitch of 4) run a thread per 16
 * sites with 16-byte row and draw accesses; the others a thread per site.
 * The result is the same. */
int prng_ising_half_sweep(const prng_ising_req *reqs, uint32_t n, void *stream);

/* Fused half-sweep (the paper's "virtualised" generator, Section 3.1: draws
 * consumed where they are made, never stored): one half-sweep of colour
 * `colour` of the L x L lattice d_spins, site of colour rank k taking draw
 * k of the handle's next stream-major block of L*L/2 draws (n_per_stream =
 * L*L/(2 n_streams) per stream), which also advances the handle.  The
 * lattice ends bit-identical to prng_fill_u32 of that block followed by
 * prng_ising_half_sweep with the generator's shift (7 for GGL and RANECU, 8
 * for XOR128 and MT19937, 0 for RANMAR and RANLUX).  L even, 2 <= L <=
 * 65534, L*L/2 a multiple of n_streams (PRNG_ESIZE otherwise).  With L a
 * multiple of 8 and d_spins 8-byte aligned, four 4-aligned colour ranks
 * update as one 8-byte chunk of their row. */
int prng_ising_fused(prng_state *st, int8_t *d_spins, uint32_t L, uint32_t colour, uint32_t t4,
                     uint32_t t8, void *stream);

/* t4 = floor(2^24 exp(-4 beta)), t8 = floor(2^24 exp(-8 beta)), in double. */
int prng_ising_thresholds(double beta, uint32_t *t4, uint32_t *t8);

/* The generator's float shift sh (the f32 output is (v >> sh) 2^-24 and the
 * Ising acceptance value is v >> sh): 7 for GGL and RANECU (31-bit words),
 * 8 for XOR128 and MT19937 (32-bit words), 0 for RANMAR and RANLUX (24-bit
 * words).  PRNG_EGEN for an unknown generator, PRNG_ENULL for a NULL
 * pointer. */
int prng_float_shift(prng_gen_t gen, uint32_t *shift);

/* Batched fill that allocates nothing (no counterpart in the paper; a
 * service of this library).  It is meant for callers that must not let a
 * library allocate device memory: code running under a framework's caching
 * allocator, services that reserve all device memory up front, and loops
 * that cannot afford the synchronisation an allocation may imply.  It does
 * what prng_batch_create + one prng_batch_launch + prng_batch_destroy do
 * for the same requests -- the same draws, the same handle advance -- but
 * its descriptors, work items and work counters live in one fixed device
 * array inside the library (about 2.4 MB, held on every device that loads
 * the library until the process exits), staged through a fixed host
 * buffer, and its kernels run one after the other on `stream`.
 *   - At most PRNG_NOALLOC_MAX_REQUESTS requests and PRNG_NOALLOC_MAX_ITEMS
 *     work items (streams / 256 per re-seeded request plus, per fill, its
 *     streams / 4 for GGL and RANECU, / 2 for MT19937, / the tile width
 *     otherwise); larger batches return PRNG_ESCRATCH and launch nothing.
 *   - The first call on a device looks up the array's device address with
 *     that device current.
 *   - Every call shares the array and the previous call's contents remain
 *     there (the work counters are cleared at the start of each call): two
 *     calls whose work overlaps on the GPU -- for example calls on two
 *     streams that nothing orders -- race and give wrong output.  Host
 *     threads are serialised by a lock around the host-side staging.
 *   - The host copy of the descriptors is pageable: the call returns once
 *     it has been handed to the device copy engine, which may wait for
 *     `stream` to drain first.
 *   - The handles' positions move only once every copy and launch of the
 *     call has been enqueued; a call that returns an error leaves every
 *     handle where it was (outputs may then be partly written). */
#define PRNG_NOALLOC_MAX_REQUESTS 4096u
#define PRNG_NOALLOC_MAX_ITEMS 131072u
int prng_batch_fill_noalloc(const prng_fill_req *reqs, uint32_t n_reqs, void *stream);

/* Measurement aid for the RANLUX roofline (no counterpart in the paper):
 * runs the RANLUX kernels' own 24-step subtract-with-borrow chain (24
 * subtract-with-borrow steps, 24 low-byte clears, 3 instructions moving the
 * borrow in and out of the carry flag: 51 integer instructions; Appendix A,
 * "AWC and SWB") `iters` times on each of `chains` (1, 2 or 4) independent
 * 24-word rings per thread, in 128-thread blocks, one wave:
 * ceil(warps_per_sm / 4) blocks per SM, or as many as fit when
 * warps_per_sm = 0.  *ops receives the integer instructions the launch
 * executes; d_sink (sink_words uint32 of device memory, at least one per
 * thread launched, else PRNG_ESIZE) receives one checksum word per thread.
 * Asynchronous on `stream`; time it with events to get the chain's
 * throughput (many chains, full occupancy) or its latency (one chain, one
 * warp per scheduler). */
int prng_calib_swb(uint32_t chains, uint32_t warps_per_sm, uint32_t iters, uint32_t *d_sink,
                   uint64_t sink_words, uint64_t *ops, void *stream);

/* Launch tile used by fills of generator `gen` (for RANLUX: of luxury p)
 * on this process: threads per CTA, staged draws per thread per tile
 * (RANMAR: 97, MT19937: 624) and staging buffers (1 or 2; for MT19937 the
 * streams per warp: 1, or 2 on half a warp each).  Set by the
 * autotuner; only the combinations compiled into the library are accepted
 * (PRNG_EUNSUPPORTED otherwise).  Not thread-safe against concurrent fills. */
int prng_set_tile(prng_gen_t gen, uint32_t luxury, uint32_t threads, uint32_t cols,
                  uint32_t stages);
int prng_get_tile(prng_gen_t gen, uint32_t luxury, uint32_t *threads, uint32_t *cols,
                  uint32_t *stages);

/* Host output buffers.  prng_host_alloc returns `bytes` of page-locked host
 * memory mapped into the device's address space at the same address
 * (unified addressing), so that the pointer can be passed as the d_out of
 * any fill, jump fill or batched request: the kernels then store the
 * numbers straight into host memory over the host link (NVLink-C2C on
 * Grace-Blackwell), with no device staging buffer and no copy.  The caller
 * owns the memory and reads it after the fill's stream has been
 * synchronised.  PRNG_ENULL if h_out is NULL, PRNG_ESIZE for bytes = 0,
 * PRNG_EALLOC if the allocation fails, PRNG_ECUDA if the device address
 * differs from the host address (no unified addressing; nothing is kept).
 * prng_host_free accepts NULL and only pointers from prng_host_alloc. */
int prng_host_alloc(void **h_out, size_t bytes);
int prng_host_free(void *h_buf);

/* Handle properties (any pointer may be NULL). */
int prng_info(const prng_state *st, int32_t *gen, int32_t *p, uint32_t *n_streams,
              uint64_t *state_bytes);

/* Release the handle's device memory.  NULL is accepted. */
void prng_destroy(prng_state *st);

/* Static English text for an error code. */
const char *prng_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* PRNG_H */
