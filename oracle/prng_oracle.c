/*
 * prng_oracle.c -- reference oracle (TEST INFRASTRUCTURE, not the library).
 *
 * Plain single-threaded C written from the definitions in V. Demchik,
 * "Pseudo-random number generators for Monte Carlo simulations on GPUs"
 * (arXiv:1003.1898), Section 3 (constants of each generator) and Appendix A
 * (the recurrences).  Each function names the passage it follows.  It is
 * deliberately written in the paper's own arithmetic (Schrage decomposition,
 * 1-based RANMAR indices, an in-place sequential Mersenne twist, ...) and
 * shares nothing with the CUDA library, which takes other arithmetic routes
 * to the same integers.
 *
 * Readings where the paper is silent or ambiguous (each is listed in the
 * design notes with its justification):
 *   R1  seeding: stream i of a handle with base seed S uses
 *       s = splitmix64(S + i), mapped per generator in orc_stream_seed().
 *   R2  XOR128: the last line of the scalar form uses the previous newest word
 *       (the matrix form in Appendix A, "XORShift", fixes this).
 *   R3  RCARRY/RANLUX: the "second variant" of SWB with the lags swapped,
 *       x_n = x_{n-10} - x_{n-24} - c, which Appendix A ("AWC and SWB")
 *       mentions and which the published RANLUX uses.
 *   R4  RANLUX: 24 numbers delivered, then p-24 discarded, p in
 *       {24,48,97,223,389} (Appendix A, "RANLUX" luxury levels), delivering
 *       the first 24 straight after seeding.  Outputs are plain 24-bit
 *       integers.
 *   R5  RMARIN (not printed in the paper) follows James (1988), which the
 *       paper cites for it, in exact integer form.
 *   R6  MT19937 initialisation (not printed) is the standard single-seed
 *       init_genrand recurrence.
 *   R7  float outputs are exact scalings (v >> sh) * 2^-24 instead of the
 *       paper's divisions by 2147483647.0 / 4294967295.0, which can round up
 *       to 1.0.
 *   R8  RANECU combination: z = s1 - s2, z += m1 - 1 when z < 1.
 */
#include "prng_oracle.h"

#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- seeding */

/* SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
 * generators", 2014): advance the state by the golden gamma, then apply the
 * mix64 finaliser (xor-shift 30, multiply, xor-shift 27, multiply,
 * xor-shift 31). */
uint64_t orc_splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* ---------------------------------------------------------------- GGL */

/* Section 3.2: m = 2147483647, a = 16807, q = 127773, r = 2836 (Park and
 * Miller's "Integer version 2").  Appendix A, "Linear congruential
 * generators": X_n = 16807 X_{n-1} mod 2147483647, evaluated without
 * overflow by the decomposition of Appendix A, "Multiple recursive
 * generators" (eq. RANECU1): a (X mod q) - floor(X/q) r, plus m if negative. */
void orc_ggl_init(orc_ggl *s, uint32_t x0) { s->x = x0; }

uint32_t orc_ggl_next(orc_ggl *s) {
  const int32_t m = 2147483647, a = 16807, q = 127773, r = 2836;
  int32_t x = (int32_t)s->x;
  int32_t t = a * (x % q) - (x / q) * r;
  if (t < 0) t += m;
  s->x = (uint32_t)t;
  return s->x;
}

/* ---------------------------------------------------------------- XOR128 */

/* Appendix A, "XORShift" (scalar form of XOR128, shifts 11/19/8 as in
 * Section 3.3):  t = X_{n-4} ^ (X_{n-4} << 11); shift the window;
 * X_n = (X_{n-1} ^ (X_{n-1} >> 19)) ^ (t ^ (t >> 8)).  Reading R2. */
void orc_xor128_init(orc_xor128 *s, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
  s->x = x; s->y = y; s->z = z; s->w = w;
}

uint32_t orc_xor128_next(orc_xor128 *s) {
  uint32_t t = s->x ^ (s->x << 11);
  uint32_t prev = s->w;                  /* X_{n-1} */
  s->x = s->y;
  s->y = s->z;
  s->z = s->w;
  s->w = (prev ^ (prev >> 19)) ^ (t ^ (t >> 8));
  return s->w;
}

/* ---------------------------------------------------------------- RANECU */

/* Section 3.4 constants; Appendix A, "Multiple recursive generators":
 * two MLCGs (a1 = 40014, m1 = 2147483563; a2 = 40692, m2 = 2147483399), each
 * evaluated by the decomposition with q = floor(m/a), r = m mod a
 * (q1 = 53668, r1 = 12211, q2 = 52774, r2 = 3791), combined as
 * (X_1 - X_2) mod (m1 - 1), plus (m1 - 1) when the result is not positive
 * (reading R8). */
void orc_ranecu_init(orc_ranecu *s, int32_t s1, int32_t s2) { s->s1 = s1; s->s2 = s2; }

uint32_t orc_ranecu_comp1(int32_t *s1) {
  int32_t k = *s1 / 53668;
  *s1 = 40014 * (*s1 - k * 53668) - k * 12211;
  if (*s1 < 0) *s1 += 2147483563;
  return (uint32_t)*s1;
}

uint32_t orc_ranecu_comp2(int32_t *s2) {
  int32_t k = *s2 / 52774;
  *s2 = 40692 * (*s2 - k * 52774) - k * 3791;
  if (*s2 < 0) *s2 += 2147483399;
  return (uint32_t)*s2;
}

uint32_t orc_ranecu_next(orc_ranecu *s) {
  orc_ranecu_comp1(&s->s1);
  orc_ranecu_comp2(&s->s2);
  int32_t z = s->s1 - s->s2;
  if (z < 1) z += 2147483562;
  return (uint32_t)z;
}

/* ---------------------------------------------------------------- RANMAR */

/* RMARIN (reading R5): James, "A review of pseudorandom number generators"
 * (1988), cited by Section 3.5 for the lag-table initialisation.  Seeds
 * ij in [0, 31328], kl in [0, 30081] (Section 3.5).  Each of the 97 table
 * entries takes 24 bits, most significant first, from a lagged 3-term
 * product generator mod 179 combined with an LCG mod 169.  The table is
 * kept in units of 2^-24 (exact, since every entry is a 24-bit binary
 * fraction). */
void orc_rmarin(orc_ranmar *s, int32_t ij, int32_t kl) {
  int32_t i = (ij / 177) % 177 + 2;
  int32_t j = ij % 177 + 2;
  int32_t k = (kl / 169) % 178 + 1;
  int32_t l = kl % 169;
  for (int ii = 1; ii <= 97; ii++) {
    int32_t acc = 0;
    int32_t bit = 1 << 23;
    for (int jj = 0; jj < 24; jj++) {
      int32_t m = (((i * j) % 179) * k) % 179;
      i = j;
      j = k;
      k = m;
      l = (53 * l + 1) % 169;
      if ((l * m) % 64 >= 32) acc += bit;
      bit >>= 1;
    }
    s->u[ii] = acc;
  }
  s->u[0] = 0;
  s->c = 362436;          /* 362436 / 2^24 */
  s->i97 = 97;
  s->j97 = 33;
}

/* Section 3.5 constants (RM_CD = 7654321/2^24, RM_CM = 16777213/2^24) and
 * Appendix A, "RANMAR": Y_n = (Y_{n-97} - Y_{n-33}) mod 2^24,
 * C_n = (C_{n-1} - D) mod M with D = 7654321, M = 2^24 - 3, and
 * X_n = (Y_n - C_n) mod 2^24 (add 2^24 when negative).  The lags are walked
 * with the two descending table indices (97, 33). */
uint32_t orc_ranmar_next(orc_ranmar *s) {
  int32_t uni = s->u[s->i97] - s->u[s->j97];
  if (uni < 0) uni += 16777216;
  s->u[s->i97] = uni;
  s->i97 -= 1;
  if (s->i97 == 0) s->i97 = 97;
  s->j97 -= 1;
  if (s->j97 == 0) s->j97 = 97;
  s->c -= 7654321;
  if (s->c < 0) s->c += 16777213;
  uni -= s->c;
  if (uni < 0) uni += 16777216;
  return (uint32_t)uni;
}

/* ---------------------------------------------------------------- RANLUX */

/* Luxury level -> p (Appendix A, "RANLUX": levels 0..4 are p = 24, 48, 97,
 * 223, 389).  p itself is accepted too, and so are the p of Section 3.6's
 * planar scheme, which discards a multiple of 24 after each 24 delivered
 * numbers (24, 96, 216, 384 at levels 1..4): p = 48, 120, 240, 408. */
int32_t orc_luxury_p(int32_t luxury) {
  static const int32_t P[5] = {24, 48, 97, 223, 389};
  static const int32_t PLANAR[3] = {120, 240, 408};
  if (luxury >= 0 && luxury <= 4) return P[luxury];
  for (int i = 0; i < 5; i++)
    if (luxury == P[i]) return luxury;
  for (int i = 0; i < 3; i++)
    if (luxury == PLANAR[i]) return luxury;
  return -1;
}

/* Seeding of the RCARRY table (the paper leaves it to a stand-alone
 * procedure, Section 3.6): an MLCG x <- 40014 x mod 2147483563 from the
 * seed, the i-th table word being the i-th LCG output mod 2^24, oldest
 * first; the initial carry is 1 only when the newest word is 0. */
void orc_ranlux_init(orc_ranlux *s, uint32_t seed, int32_t p) {
  int32_t lcg = (int32_t)(seed % 2147483563u);
  if (lcg == 0) lcg = 1;
  for (int i = 0; i < 24; i++) {
    orc_ranecu_comp1(&lcg);   /* same MLCG as RANECU's first component */
    s->x[i] = lcg % 16777216;
  }
  s->k = 0;                   /* x[k] holds x_{n-24}, the oldest word */
  s->carry = (s->x[23] == 0) ? 1 : 0;
  s->p = p;
  s->pos = 0;
}

/* Appendix A, "AWC and SWB" (eq. RCARRY) with m = 2^24, r = 24, s = 10 in
 * the swapped variant (reading R3):
 *   t = x_{n-10} - x_{n-24} - c_{n-1};  c_n = (t < 0);  x_n = t mod 2^24. */
uint32_t orc_swb_step(orc_ranlux *s) {
  int32_t oldest = s->x[s->k];                  /* x_{n-24} */
  int32_t lag10 = s->x[(s->k + 14) % 24];       /* x_{n-10} */
  int32_t t = lag10 - oldest - s->carry;
  if (t < 0) {
    t += 16777216;
    s->carry = 1;
  } else {
    s->carry = 0;
  }
  s->x[s->k] = t;
  s->k = (s->k + 1) % 24;
  return (uint32_t)t;
}

/* Appendix A, "RANLUX": after delivering r = 24 values, the next p - 24
 * core values are discarded (reading R4). */
uint32_t orc_ranlux_next(orc_ranlux *s) {
  if (s->pos == 24) {
    for (int i = 0; i < s->p - 24; i++) orc_swb_step(s);
    s->pos = 0;
  }
  s->pos += 1;
  return orc_swb_step(s);
}

/* ---------------------------------------------------------------- MT19937 */

/* Single-seed initialisation (reading R6): mt[0] = seed,
 * mt[i] = 1812433253 (mt[i-1] ^ (mt[i-1] >> 30)) + i  (mod 2^32). */
void orc_mt_init(orc_mt *s, uint32_t seed) {
  s->mt[0] = seed;
  for (int i = 1; i < 624; i++)
    s->mt[i] = 1812433253u * (s->mt[i - 1] ^ (s->mt[i - 1] >> 30)) + (uint32_t)i;
  s->mti = 624;
}

/* Appendix A, "Mersenne twister": X_{n+r} = X_{n+s} ^ (X_n^upper | X_{n+1}^lower) A
 * with w = 32, r = 624, s = 397, u = 31, a = 0x9908B0DF; X A = X >> 1, xor a
 * when the low bit of X is set.  Applied in place for n = 0..623 in order,
 * so that entries from 227 on see the words already replaced.  Tempering
 * with (11; 7, 0x9D2C5680; 15, 0xEFC60000; 18) as in Section 3.7. */
static void orc_mt_twist(orc_mt *s) {
  for (int n = 0; n < 624; n++) {
    uint32_t y = (s->mt[n] & 0x80000000u) | (s->mt[(n + 1) % 624] & 0x7FFFFFFFu);
    uint32_t ya = y >> 1;
    if (y & 1u) ya ^= 0x9908B0DFu;
    s->mt[n] = s->mt[(n + 397) % 624] ^ ya;
  }
  s->mti = 0;
}

uint32_t orc_mt_next(orc_mt *s) {
  if (s->mti >= 624) orc_mt_twist(s);
  uint32_t t = s->mt[s->mti++];
  t ^= t >> 11;
  t ^= (t << 7) & 0x9D2C5680u;
  t ^= (t << 15) & 0xEFC60000u;
  t ^= t >> 18;
  return t;
}

/* ---------------------------------------------------------------- floats */

/* Reading R7: exact float = (v >> sh) 2^-24, computed in double and
 * narrowed (the value has at most 24 significant bits, so both steps are
 * exact). */
float orc_to_f32(int32_t gen, uint32_t v) {
  int sh = 0;
  if (gen == ORC_GGL || gen == ORC_RANECU) sh = 7;
  else if (gen == ORC_XOR128 || gen == ORC_MT19937) sh = 8;
  double d = (double)(v >> sh) / 16777216.0;
  return (float)d;
}

/* Reading R11: a double from two consecutive draws (Section 3.1 and
 * Section 4 ask for doubles built from several draws rather than a widened
 * single one, without a rule).  The high part comes from the first draw a,
 * the low part from the second draw b, both taken from the top of the
 * generator's word:
 *   24-bit words (RANMAR, RANLUX): (a 2^24 + b) 2^-48;
 *   31-bit words (GGL, RANECU):    ((a >> 4) 2^26 + (b >> 5)) 2^-53;
 *   32-bit words (XOR128, MT19937): ((a >> 5) 2^26 + (b >> 6)) 2^-53.
 * The integer has at most 53 bits and the scale is a power of two, so the
 * value is exact and lies in [0, 1). */
double orc_to_f64(int32_t gen, uint32_t a, uint32_t b) {
  if (gen == ORC_RANMAR || gen == ORC_RANLUX)
    return ((double)a * 16777216.0 + (double)b) / 281474976710656.0;
  int sa = 5, sb = 6;
  if (gen == ORC_GGL || gen == ORC_RANECU) { sa = 4; sb = 5; }
  return ((double)(a >> sa) * 67108864.0 + (double)(b >> sb)) / 9007199254740992.0;
}

/* ---------------------------------------------------------------- streams */

/* Reading R1: s = splitmix64(seed + i), then
 *   GGL     x0 = 1 + s mod (2^31 - 2)
 *   XOR128  (x, y) = (lo32 s, hi32 s), (z, w) = (lo32 t, hi32 t), t = splitmix64(s);
 *           w = 1 if all four are zero
 *   RANECU  s1 = 1 + lo32(s) mod (m1 - 1), s2 = 1 + hi32(s) mod (m2 - 1)
 *   RANMAR  ij = lo32(s) mod 31329, kl = hi32(s) mod 30082
 *   RANLUX  j = s mod 2147483563, 19780503 when that is 0
 *   MT19937 seed = lo32(s) */
int orc_stream_seed(orc_stream *st, int32_t gen, int32_t luxury, uint64_t seed, uint64_t i) {
  uint64_t s = orc_splitmix64(seed + i);
  uint32_t lo = (uint32_t)s, hi = (uint32_t)(s >> 32);
  memset(st, 0, sizeof(*st));
  st->gen = gen;
  switch (gen) {
    case ORC_GGL:
      orc_ggl_init(&st->s.g, (uint32_t)(1 + s % 2147483646ull));
      return 0;
    case ORC_XOR128: {
      uint64_t t = orc_splitmix64(s);
      uint32_t z = (uint32_t)t, w = (uint32_t)(t >> 32);
      if (lo == 0 && hi == 0 && z == 0 && w == 0) w = 1;
      orc_xor128_init(&st->s.x, lo, hi, z, w);
      return 0;
    }
    case ORC_RANECU:
      orc_ranecu_init(&st->s.e, (int32_t)(1 + lo % 2147483562u),
                      (int32_t)(1 + hi % 2147483398u));
      return 0;
    case ORC_RANMAR:
      orc_rmarin(&st->s.m, (int32_t)(lo % 31329u), (int32_t)(hi % 30082u));
      return 0;
    case ORC_RANLUX: {
      int32_t p = orc_luxury_p(luxury);
      if (p < 0) return -1;
      uint32_t j = (uint32_t)(s % 2147483563ull);
      if (j == 0) j = 19780503u;
      orc_ranlux_init(&st->s.l, j, p);
      return 0;
    }
    case ORC_MT19937:
      orc_mt_init(&st->s.t, lo);
      return 0;
    default:
      return -1;
  }
}

uint32_t orc_stream_next(orc_stream *st) {
  switch (st->gen) {
    case ORC_GGL: return orc_ggl_next(&st->s.g);
    case ORC_XOR128: return orc_xor128_next(&st->s.x);
    case ORC_RANECU: return orc_ranecu_next(&st->s.e);
    case ORC_RANMAR: return orc_ranmar_next(&st->s.m);
    case ORC_RANLUX: return orc_ranlux_next(&st->s.l);
    case ORC_MT19937: return orc_mt_next(&st->s.t);
    default: return 0;
  }
}

int orc_fill(int32_t gen, int32_t luxury, uint64_t seed, uint64_t stream0,
             uint32_t n_streams, uint64_t skip, uint64_t n_per,
             uint32_t *out_u32, float *out_f32) {
  orc_stream st;
  for (uint64_t i = 0; i < n_streams; i++) {
    if (orc_stream_seed(&st, gen, luxury, seed, stream0 + i) != 0) return -1;
    for (uint64_t k = 0; k < skip; k++) orc_stream_next(&st);
    for (uint64_t k = 0; k < n_per; k++) {
      uint32_t v = orc_stream_next(&st);
      if (out_u32) out_u32[i * n_per + k] = v;
      if (out_f32) out_f32[i * n_per + k] = orc_to_f32(gen, v);
    }
  }
  return 0;
}

int orc_fill_f64(int32_t gen, int32_t luxury, uint64_t seed, uint64_t stream0,
                 uint32_t n_streams, uint64_t skip, uint64_t n_per, double *out) {
  orc_stream st;
  for (uint64_t i = 0; i < n_streams; i++) {
    if (orc_stream_seed(&st, gen, luxury, seed, stream0 + i) != 0) return -1;
    for (uint64_t k = 0; k < skip; k++) orc_stream_next(&st);
    for (uint64_t k = 0; k < n_per; k++) {
      uint32_t a = orc_stream_next(&st);
      uint32_t b = orc_stream_next(&st);
      out[i * n_per + k] = orc_to_f64(gen, a, b);
    }
  }
  return 0;
}

int orc_sample(int32_t gen, int32_t luxury, uint64_t seed, uint64_t stream,
               const uint64_t *pos, uint64_t n_pos, uint32_t *out_u32) {
  orc_stream st;
  if (orc_stream_seed(&st, gen, luxury, seed, stream) != 0) return -1;
  uint64_t at = 0;      /* number of draws taken so far */
  for (uint64_t i = 0; i < n_pos; i++) {
    if (i > 0 && pos[i] < pos[i - 1]) return -1;
    uint32_t v = 0;
    if (i > 0 && pos[i] == pos[i - 1]) {
      out_u32[i] = out_u32[i - 1];
      continue;
    }
    while (at <= pos[i]) {
      v = orc_stream_next(&st);
      at++;
    }
    out_u32[i] = v;
  }
  return 0;
}

int orc_explicit_draws(int32_t gen, int32_t luxury, const uint64_t *seeds,
                       uint32_t n_seeds, uint64_t n, uint32_t *out_u32) {
  static const uint32_t need[ORC_NGEN] = {1, 4, 2, 2, 1, 1};
  orc_stream st;
  if (gen < 0 || gen >= ORC_NGEN || n_seeds < need[gen]) return -1;
  memset(&st, 0, sizeof(st));
  st.gen = gen;
  switch (gen) {
    case ORC_GGL: orc_ggl_init(&st.s.g, (uint32_t)seeds[0]); break;
    case ORC_XOR128:
      orc_xor128_init(&st.s.x, (uint32_t)seeds[0], (uint32_t)seeds[1],
                      (uint32_t)seeds[2], (uint32_t)seeds[3]);
      break;
    case ORC_RANECU: orc_ranecu_init(&st.s.e, (int32_t)seeds[0], (int32_t)seeds[1]); break;
    case ORC_RANMAR: orc_rmarin(&st.s.m, (int32_t)seeds[0], (int32_t)seeds[1]); break;
    case ORC_RANLUX: {
      int32_t p = orc_luxury_p(luxury);
      if (p < 0) return -1;
      orc_ranlux_init(&st.s.l, (uint32_t)seeds[0], p);
      break;
    }
    case ORC_MT19937: orc_mt_init(&st.s.t, (uint32_t)seeds[0]); break;
  }
  for (uint64_t k = 0; k < n; k++) out_u32[k] = orc_stream_next(&st);
  return 0;
}

/* ---------------------------------------------------------------- jump-ahead */

/* Square-and-multiply; m < 2^32, so every product fits in 64 bits. */
uint64_t orc_modpow(uint64_t a, uint64_t e, uint64_t m) {
  uint64_t result = 1 % m, base = a % m;
  while (e > 0) {
    if (e & 1) result = (result * base) % m;
    base = (base * base) % m;
    e >>= 1;
  }
  return result;
}

/* MLCG in closed form (Appendix A, eq. MLCG): X_{n+k} = a^k X_n mod m. */
uint32_t orc_ggl_jump(uint32_t x, uint64_t k) {
  uint64_t ak = orc_modpow(16807, k, 2147483647);
  return (uint32_t)((ak * x) % 2147483647ull);
}

void orc_ranecu_jump(orc_ranecu *s, uint64_t k) {
  uint64_t a1 = orc_modpow(40014, k, 2147483563), a2 = orc_modpow(40692, k, 2147483399);
  s->s1 = (int32_t)((a1 * (uint64_t)s->s1) % 2147483563ull);
  s->s2 = (int32_t)((a2 * (uint64_t)s->s2) % 2147483399ull);
}

/* XOR128 jump-ahead over GF(2) (Appendix A, "XORShift", matrix form): the
 * state (x, y, z, w) is a 128-bit vector v (bit 32 i + b = bit b of word i,
 * words in the order x, y, z, w) and one step is v <- T v for the 128 x 128
 * block matrix T, so k steps are v <- T^k v.  T is taken column by column
 * from the scalar step applied to the unit vectors (column j = T e_j), and
 * T^k by square-and-multiply of 128 x 128 matrices over GF(2). */
typedef struct { uint32_t col[128][4]; } orc_gf2_128;

static void orc_gf2_apply(const orc_gf2_128 *A, const uint32_t v[4], uint32_t out[4]) {
  uint32_t r[4] = {0, 0, 0, 0};
  for (int j = 0; j < 128; j++)
    if ((v[j / 32] >> (j % 32)) & 1u)
      for (int i = 0; i < 4; i++) r[i] ^= A->col[j][i];
  for (int i = 0; i < 4; i++) out[i] = r[i];
}

static void orc_gf2_mul(const orc_gf2_128 *A, const orc_gf2_128 *B, orc_gf2_128 *C) {
  orc_gf2_128 t;
  for (int j = 0; j < 128; j++) orc_gf2_apply(A, B->col[j], t.col[j]);
  *C = t;
}

void orc_xor128_jump(orc_xor128 *s, uint64_t k) {
  orc_gf2_128 T, R;
  for (int j = 0; j < 128; j++) {
    orc_xor128 e;
    uint32_t unit[4] = {0, 0, 0, 0};
    unit[j / 32] = 1u << (j % 32);
    orc_xor128_init(&e, unit[0], unit[1], unit[2], unit[3]);
    orc_xor128_next(&e);
    T.col[j][0] = e.x; T.col[j][1] = e.y; T.col[j][2] = e.z; T.col[j][3] = e.w;
    for (int i = 0; i < 4; i++) R.col[j][i] = (i == j / 32) ? (1u << (j % 32)) : 0u;
  }
  while (k > 0) {  /* R = T^k */
    if (k & 1) orc_gf2_mul(&T, &R, &R);
    orc_gf2_mul(&T, &T, &T);
    k >>= 1;
  }
  uint32_t v[4] = {s->x, s->y, s->z, s->w}, o[4];
  orc_gf2_apply(&R, v, o);
  s->x = o[0]; s->y = o[1]; s->z = o[2]; s->w = o[3];
}

/* XOR128 state that the stream seeding map (reading R1) gives for the
 * per-stream value s: (x, y) = (lo32 s, hi32 s), (z, w) = halves of
 * splitmix64(s), w = 1 if all four are zero. */
static void orc_xor128_from_s(orc_xor128 *x, uint64_t s) {
  uint64_t t = orc_splitmix64(s);
  uint32_t lo = (uint32_t)s, hi = (uint32_t)(s >> 32), z = (uint32_t)t, w = (uint32_t)(t >> 32);
  if (lo == 0 && hi == 0 && z == 0 && w == 0) w = 1;
  orc_xor128_init(x, lo, hi, z, w);
}

/* MT19937 jump-ahead over GF(2).  The table of 624 words is a window
 * (w_s, ..., w_{s+623}) of the word sequence of Appendix A, "Mersenne
 * twister" (w_{t+624} = w_{t+397} ^ (w_t^upper | w_{t+1}^lower) A), the
 * next outputs being tempered words of it, so k outputs later the table is
 * the window k words on (the read index mti is unchanged).  Moving the window
 * by one word is a linear map T over GF(2).  Its characteristic polynomial
 * phi, of degree 19937, is found here by the Berlekamp-Massey algorithm from
 * 2 x 19937 output bits, and on the state T^k acts as g(T) with g = t^k mod
 * phi.  T drops the low 31 bits of the window's oldest word, which are not
 * part of the state, so the window is moved by g(T) for t^(k-1) and then
 * one more word: word j of the new table is the XOR of w_{1+i+j} over the
 * coefficients g_i = 1. */
#define ORC_MT_DEG 19937
static uint8_t *orc_mt_phi;            /* coefficients of t^0 .. t^19937 */
static int32_t orc_mt_phi_exp[ORC_MT_DEG + 1];
static int32_t orc_mt_phi_nterms;

static void orc_mt_charpoly(void) {
  if (orc_mt_phi) return;
  const int32_t N = 2 * ORC_MT_DEG;
  uint8_t *seq = (uint8_t *)malloc(N), *C = (uint8_t *)calloc(N + 1, 1);
  uint8_t *B = (uint8_t *)calloc(N + 1, 1), *T = (uint8_t *)malloc(N + 1);
  orc_mt st;
  orc_mt_init(&st, 5489u);
  for (int32_t n = 0; n < N; n++) seq[n] = (uint8_t)(orc_mt_next(&st) & 1u);
  /* Berlekamp-Massey: the shortest C with sum_{i=0..L} C_i s_{n-i} = 0. */
  int32_t L = 0, m = 1;
  C[0] = B[0] = 1;
  for (int32_t n = 0; n < N; n++) {
    uint8_t d = seq[n];
    for (int32_t i = 1; i <= L; i++) d ^= (uint8_t)(C[i] & seq[n - i]);
    if (!d) {
      m++;
      continue;
    }
    if (2 * L <= n) {
      memcpy(T, C, (size_t)N + 1);
      for (int32_t i = 0; i + m <= N; i++) C[i + m] ^= B[i];
      L = n + 1 - L;
      memcpy(B, T, (size_t)N + 1);
      m = 1;
    } else {
      for (int32_t i = 0; i + m <= N; i++) C[i + m] ^= B[i];
      m++;
    }
  }
  /* phi(t) = t^L C(1/t). */
  uint8_t *phi = (uint8_t *)calloc((size_t)L + 1, 1);
  for (int32_t i = 0; i <= L; i++) phi[L - i] = C[i];
  orc_mt_phi_nterms = 0;
  for (int32_t e = 0; e <= L; e++)
    if (phi[e]) orc_mt_phi_exp[orc_mt_phi_nterms++] = e;
  free(seq); free(C); free(B); free(T);
  orc_mt_phi = phi;
}

/* Degree and number of terms of the characteristic polynomial. */
int32_t orc_mt_charpoly_info(int32_t *n_terms) {
  orc_mt_charpoly();
  if (n_terms) *n_terms = orc_mt_phi_nterms;
  return orc_mt_phi_exp[orc_mt_phi_nterms - 1];
}

/* r (coefficients 0 .. 2 D - 2) reduced mod phi in place. */
static void orc_mt_reduce(uint8_t *r, int32_t top) {
  for (int32_t p = top; p >= ORC_MT_DEG; p--) {
    if (!r[p]) continue;
    for (int32_t j = 0; j < orc_mt_phi_nterms; j++) r[p - ORC_MT_DEG + orc_mt_phi_exp[j]] ^= 1;
  }
}

void orc_mt_jump(orc_mt *s, uint64_t k) {
  if (k == 0) return;
  orc_mt_charpoly();
  const int32_t D = ORC_MT_DEG;
  uint8_t *g = (uint8_t *)calloc(2 * (size_t)D, 1), *r = (uint8_t *)calloc(2 * (size_t)D, 1);
  /* g = t^(k-1) mod phi, left to right over the bits of k - 1. */
  const uint64_t e = k - 1;
  g[0] = 1;
  for (int b = 63; b >= 0; b--) {
    memset(r, 0, 2 * (size_t)D);
    for (int32_t i = 0; i < D; i++) r[2 * i] = g[i];          /* squaring over GF(2) */
    orc_mt_reduce(r, 2 * D - 2);
    if ((e >> b) & 1u) {                                      /* times t */
      memmove(r + 1, r, (size_t)D);
      r[0] = 0;
      orc_mt_reduce(r, D);
    }
    memcpy(g, r, (size_t)D);
  }
  /* The word sequence from the table, then the new table. */
  const int32_t W = D + 624 + 1;
  uint32_t *w = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)W);
  for (int32_t j = 0; j < 624; j++) w[j] = s->mt[j];
  for (int32_t t = 0; t + 624 < W; t++) {
    uint32_t y = (w[t] & 0x80000000u) | (w[t + 1] & 0x7FFFFFFFu);
    uint32_t ya = y >> 1;
    if (y & 1u) ya ^= 0x9908B0DFu;
    w[t + 624] = w[t + 397] ^ ya;
  }
  for (int32_t j = 0; j < 624; j++) {
    uint32_t acc = 0;
    for (int32_t i = 0; i < D; i++)
      if (g[i]) acc ^= w[1 + i + j];
    s->mt[j] = acc;
  }
  free(w); free(g); free(r);
}

static int orc_serial_start(orc_stream *st, int32_t gen, uint64_t x0) {
  memset(st, 0, sizeof(*st));
  st->gen = gen;
  if (gen == ORC_GGL) {
    if (x0 == 0 || x0 >= 2147483647ull) return -1;
    orc_ggl_init(&st->s.g, (uint32_t)x0);
    return 0;
  }
  if (gen == ORC_RANECU) {
    uint64_t s1 = x0 & 0xFFFFFFFFull, s2 = x0 >> 32;
    if (s1 == 0 || s1 >= 2147483563ull || s2 == 0 || s2 >= 2147483399ull) return -1;
    orc_ranecu_init(&st->s.e, (int32_t)s1, (int32_t)s2);
    return 0;
  }
  if (gen == ORC_XOR128) {
    orc_xor128_from_s(&st->s.x, x0);
    return 0;
  }
  if (gen == ORC_MT19937) {
    if (x0 > 0xFFFFFFFFull) return -1;
    orc_mt_init(&st->s.t, (uint32_t)x0);
    return 0;
  }
  return -1;
}

int orc_serial_sample(int32_t gen, uint64_t x0, const uint64_t *pos,
                      uint64_t n_pos, uint32_t *out_u32) {
  orc_stream st;
  if (orc_serial_start(&st, gen, x0) != 0) return -1;
  uint64_t at = 0;
  uint32_t v = 0;
  for (uint64_t i = 0; i < n_pos; i++) {
    if (i > 0 && pos[i] < pos[i - 1]) return -1;
    while (at <= pos[i]) {
      v = orc_stream_next(&st);
      at++;
    }
    out_u32[i] = v;
  }
  return 0;
}

int orc_serial_fill(int32_t gen, uint64_t x0, uint64_t n, uint32_t *out_u32) {
  orc_stream st;
  if (orc_serial_start(&st, gen, x0) != 0) return -1;
  for (uint64_t j = 0; j < n; j++) out_u32[j] = orc_stream_next(&st);
  return 0;
}

/* ---------------------------------------------------------------- Ising */

void orc_ising_thresholds(double beta, uint32_t *t4, uint32_t *t8) {
  *t4 = (uint32_t)floor(16777216.0 * exp(-4.0 * beta));
  *t8 = (uint32_t)floor(16777216.0 * exp(-8.0 * beta));
}

void orc_ising_half_sweep(int32_t L, int8_t *spins, const uint32_t *draws, int32_t shift,
                          uint32_t t4, uint32_t t8, int32_t colour) {
  for (int32_t y = 0; y < L; y++) {
    for (int32_t x = 0; x < L; x++) {
      if ((x + y) % 2 != colour) continue;
      int32_t k = y * (L / 2) + x / 2;
      int32_t s = spins[y * L + x];
      int32_t up = spins[((y + L - 1) % L) * L + x];
      int32_t down = spins[((y + 1) % L) * L + x];
      int32_t left = spins[y * L + (x + L - 1) % L];
      int32_t right = spins[y * L + (x + 1) % L];
      int32_t dE = 2 * s * (up + down + left + right);
      uint32_t r = draws[k] >> shift;
      int accept;
      if (dE <= 0) accept = 1;
      else if (dE == 4) accept = r < t4;
      else accept = r < t8;
      if (accept) spins[y * L + x] = (int8_t)(-s);
    }
  }
}

int64_t orc_ising_energy(int32_t L, const int8_t *spins) {
  int64_t e = 0;
  for (int32_t y = 0; y < L; y++)
    for (int32_t x = 0; x < L; x++) {
      int32_t s = spins[y * L + x];
      e -= s * spins[y * L + (x + 1) % L];
      e -= s * spins[((y + 1) % L) * L + x];
    }
  return e;
}

int64_t orc_ising_magnetisation(int32_t L, const int8_t *spins) {
  int64_t m = 0;
  for (int64_t i = 0; i < (int64_t)L * L; i++) m += spins[i];
  return m;
}

/* ---------------------------------------------------------------- timing */

/* The paper's CPU measurement (Section 4): one generator call per number,
 * summed so the work stays observable. */
uint64_t orc_checksum_draws(int32_t gen, int32_t luxury, uint64_t seed,
                            uint64_t stream, uint64_t n) {
  orc_stream st;
  if (orc_stream_seed(&st, gen, luxury, seed, stream) != 0) return 0;
  uint64_t sum = 0;
  for (uint64_t k = 0; k < n; k++) sum += orc_stream_next(&st);
  return sum;
}
