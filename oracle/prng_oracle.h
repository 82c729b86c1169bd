/*
 * prng_oracle.h -- reference oracle for the six uniform generators of
 * V. Demchik, "Pseudo-random number generators for Monte Carlo simulations
 * on Graphics Processing Units" (arXiv:1003.1898).
 *
 * TEST INFRASTRUCTURE, NOT PART OF THE LIBRARY.  Plain, slow, single-threaded
 * C written from the paper's definitions.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg load it.  It shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * Conventions
 *   - A generator "draw" is one delivered output.  Draw n is 1-based: the
 *     first value returned after seeding is draw 1.
 *   - u32 outputs: GGL x_n in [1, 2^31-2]; XOR128 the new word w; RANECU the
 *     combined z in [1, 2147483562]; RANMAR and RANLUX the 24-bit integer
 *     (the paper's float value times 2^24); MT19937 the tempered word.
 *   - f32 outputs are (v >> sh) * 2^-24 computed exactly, with sh = 7 for
 *     GGL/RANECU, 8 for XOR128/MT19937 and 0 for RANMAR/RANLUX.
 *
 * Parity pins live in tests/test_oracle_pins.py.  The RANECU combination
 * step, for which no printed value exists, is pinned at the boundaries of
 * its rule (equal components, differences of -1 and 1, components at their
 * extremes; tests/golden/ranecu_combination.txt) and by the congruence
 * Z = X1 - X2 (mod m1 - 1) with Z in [1, m1 - 1].  XOR128, which has no
 * known answer in the paper, is pinned by its GF(2) matrix form, by
 * linearity and by the outputs of Marsaglia's routine from its published
 * initial state.
 */
#ifndef PRNG_ORACLE_H
#define PRNG_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Generator ids used by this oracle (its own numbering). */
enum { ORC_GGL = 0, ORC_XOR128 = 1, ORC_RANECU = 2, ORC_RANMAR = 3,
       ORC_RANLUX = 4, ORC_MT19937 = 5, ORC_NGEN = 6 };

typedef struct { uint32_t x; } orc_ggl;
typedef struct { uint32_t x, y, z, w; } orc_xor128;
typedef struct { int32_t s1, s2; } orc_ranecu;
typedef struct { int32_t u[98]; int32_t c; int32_t i97, j97; } orc_ranmar;
typedef struct { int32_t x[24]; int32_t k; int32_t carry; int32_t p; int32_t pos; } orc_ranlux;
typedef struct { uint32_t mt[624]; int32_t mti; } orc_mt;

/* One stream of any generator. */
typedef struct {
  int32_t gen;
  union { orc_ggl g; orc_xor128 x; orc_ranecu e; orc_ranmar m; orc_ranlux l; orc_mt t; } s;
} orc_stream;

/* SplitMix64 (Steele, Lea, Flood 2014): first output of a SplitMix64
 * generator whose state is x. */
uint64_t orc_splitmix64(uint64_t x);

/* Per-generator initialisation from explicit seeds. */
void orc_ggl_init(orc_ggl *s, uint32_t x0);
void orc_xor128_init(orc_xor128 *s, uint32_t x, uint32_t y, uint32_t z, uint32_t w);
void orc_ranecu_init(orc_ranecu *s, int32_t s1, int32_t s2);
void orc_rmarin(orc_ranmar *s, int32_t ij, int32_t kl);
void orc_ranlux_init(orc_ranlux *s, uint32_t seed, int32_t p);
void orc_mt_init(orc_mt *s, uint32_t seed);

/* One draw. */
uint32_t orc_ggl_next(orc_ggl *s);
uint32_t orc_xor128_next(orc_xor128 *s);
uint32_t orc_ranecu_next(orc_ranecu *s);
uint32_t orc_ranecu_comp1(int32_t *s1);   /* first MLCG component alone */
uint32_t orc_ranecu_comp2(int32_t *s2);   /* second MLCG component alone */
uint32_t orc_ranmar_next(orc_ranmar *s);
uint32_t orc_swb_step(orc_ranlux *s);     /* one RCARRY core step, no decimation */
uint32_t orc_ranlux_next(orc_ranlux *s);
uint32_t orc_mt_next(orc_mt *s);

/* Luxury level 0..4 or p in {24,48,97,223,389} -> p; -1 if invalid. */
int32_t orc_luxury_p(int32_t luxury);

/* Exact float conversion of a u32 output of generator gen. */
float orc_to_f32(int32_t gen, uint32_t v);

/* Seed stream i of a handle created with base seed `seed`:
 * s = splitmix64(seed + i), then the per-generator map.  Returns 0 or -1. */
int orc_stream_seed(orc_stream *st, int32_t gen, int32_t luxury, uint64_t seed, uint64_t i);
uint32_t orc_stream_next(orc_stream *st);

/* Reading R11: the double made of the consecutive draws a then b (24-bit
 * words: (a 2^24 + b) 2^-48; 31-bit: ((a >> 4) 2^26 + (b >> 5)) 2^-53;
 * 32-bit: ((a >> 5) 2^26 + (b >> 6)) 2^-53), exact, in [0, 1). */
double orc_to_f64(int32_t gen, uint32_t a, uint32_t b);
/* Doubles of streams [stream0, stream0+n_streams) after `skip` draws:
 * out[i n_per + k] = orc_to_f64 of draws 2k+1 and 2k+2 after the skip. */
int orc_fill_f64(int32_t gen, int32_t luxury, uint64_t seed, uint64_t stream0,
                 uint32_t n_streams, uint64_t skip, uint64_t n_per, double *out);

/* Streams [stream0, stream0+n_streams) of a handle (gen, luxury, seed): each
 * stream first discards `skip` draws, then writes n_per draws, stream-major.
 * Either output pointer may be NULL.  Returns 0 or -1. */
int orc_fill(int32_t gen, int32_t luxury, uint64_t seed, uint64_t stream0,
             uint32_t n_streams, uint64_t skip, uint64_t n_per,
             uint32_t *out_u32, float *out_f32);

/* Draws at sorted 0-based positions pos[0..n_pos) of one stream. */
int orc_sample(int32_t gen, int32_t luxury, uint64_t seed, uint64_t stream,
               const uint64_t *pos, uint64_t n_pos, uint32_t *out_u32);

/* n draws of a stream initialised from explicit seeds instead of the
 * splitmix64 map: GGL {x0}; XOR128 {x,y,z,w}; RANECU {s1,s2}; RANMAR
 * {ij,kl}; RANLUX {seed} with the given luxury; MT19937 {seed}.
 * Returns 0 or -1. */
int orc_explicit_draws(int32_t gen, int32_t luxury, const uint64_t *seeds,
                       uint32_t n_seeds, uint64_t n, uint32_t *out_u32);

/* Modular exponentiation a^e mod m by square-and-multiply (m < 2^32). */
uint64_t orc_modpow(uint64_t a, uint64_t e, uint64_t m);

/* Jump-ahead of the multiplicative congruential generators:
 * x_{n+k} = (a^k mod m) x_n mod m, applied to GGL and to each RANECU
 * component separately. */
uint32_t orc_ggl_jump(uint32_t x, uint64_t k);
void orc_ranecu_jump(orc_ranecu *s, uint64_t k);
/* XOR128 jump-ahead: the state after k steps, T^k v over GF(2) with T the
 * 128 x 128 matrix of one step (Appendix A, "XORShift", matrix form). */
void orc_xor128_jump(orc_xor128 *s, uint64_t k);
/* MT19937 jump-ahead: the state k outputs later (the table moved k words on
 * along the word sequence, mti unchanged), by g(T) with g = t^(k-1) mod phi
 * and one more step; phi, the characteristic polynomial of the one-word
 * step T, comes from Berlekamp-Massey on 2 x 19937 output bits. */
void orc_mt_jump(orc_mt *s, uint64_t k);
/* Degree of phi; *n_terms receives its number of nonzero coefficients. */
int32_t orc_mt_charpoly_info(int32_t *n_terms);

/* The single serial sequence started at x0 (GGL: x0 = seed value; RANECU:
 * x0 = s1 | s2 << 32; XOR128: the state the stream seeding map gives for the
 * per-stream value s = x0; MT19937: init_genrand(x0), x0 < 2^32):
 * out[j] = draw j+1.  Returns the draws at sorted
 * 0-based positions pos[0..n_pos) by stepping serially. */
int orc_serial_sample(int32_t gen, uint64_t x0, const uint64_t *pos,
                      uint64_t n_pos, uint32_t *out_u32);
/* Same sequence, the first n draws, written in full. */
int orc_serial_fill(int32_t gen, uint64_t x0, uint64_t n, uint32_t *out_u32);

/* ------------------------------------------------------------ Ising consumer
 * Checkerboard Metropolis half-sweep of the periodic L x L Ising model
 * (J = 1, h = 0), the Monte Carlo use the paper's generators serve (Section
 * 3.5 cites RANMAR's earlier use for Ising simulations).  Spins are +1/-1 in
 * int8, row-major.  Only sites of colour `colour` ((x + y) % 2) are
 * visited; the site with colour rank k (row-major order among sites of that
 * colour, k = y L/2 + x/2) uses draw draws[k], whose 24-bit value
 * r = draws[k] >> shift is compared with the integer thresholds:
 * the flip is accepted when dE = 2 s (sum of the 4 neighbours) <= 0, or
 * when r < t4 (dE = 4) or r < t8 (dE = 8).  L must be even. */
void orc_ising_half_sweep(int32_t L, int8_t *spins, const uint32_t *draws, int32_t shift,
                          uint32_t t4, uint32_t t8, int32_t colour);
/* floor(2^24 exp(-dE beta)) for dE = 4 and 8, evaluated in double. */
void orc_ising_thresholds(double beta, uint32_t *t4, uint32_t *t8);
/* E = -sum over nearest-neighbour bonds of s_i s_j (each bond once). */
int64_t orc_ising_energy(int32_t L, const int8_t *spins);
int64_t orc_ising_magnetisation(int32_t L, const int8_t *spins);

/* Timing helper for the CPU baseline: draws n values from one stream and
 * returns a running checksum so the work cannot be optimised away. */
uint64_t orc_checksum_draws(int32_t gen, int32_t luxury, uint64_t seed,
                            uint64_t stream, uint64_t n);

#ifdef __cplusplus
}
#endif
#endif
