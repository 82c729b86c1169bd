// k_mt.cu -- MT19937 fill and skip (Section 3.7; Appendix A, "Mersenne
// twister").
//
// A warp per stream (or half a warp, two streams per warp), its 624-word
// table in shared memory.  The twist X_{n+624} = X_{n+397} ^ (X_n^upper |
// X_{n+1}^lower) A is done in place in five chunks of 128 consecutive
// entries, in increasing order: entry k reads old k and k+1 and either old
// k+397 (k < 227) or new k-227 (k >= 227, produced in an earlier chunk), so
// a chunk needs only a __syncwarp between its reads and its writes.  Each
// new word is tempered and stored by the lane that produced it: a lane's 4
// words are 16 bytes of a run of 512 (a warp) or 256 (a half) consecutive
// bytes of the stream's row, written without staging.  In the fill kernels
// a lane keeps its own quads of the table in registers from one 624-word
// block to the next (mt_blocks_reg), so the shared table serves only the
// other lanes' lag reads (the batched kernel keeps the shared-table form).
// What bounds the kernel is then the integer ALU: the twist's and the
// tempering's logic instructions.
#include "batch.cuh"

namespace prng {

// The tempering's left shifts, 7 and 15, as multiplies by 2^7 and 2^15 from
// the constant bank: they then run on the FMA pipe rather than the integer
// ALU, which the twist and the right shifts keep busy.
__constant__ uint32_t c_mt_shl[2] = {1u << 7, 1u << 15};

__device__ __forceinline__ uint32_t mt_temper(uint32_t t) {
  t ^= t >> 11;
  t ^= (t * c_mt_shl[0]) & 0x9D2C5680u;
  t ^= (t * c_mt_shl[1]) & 0xEFC60000u;
  t ^= t >> 18;
  return t;
}

// Float of a tempered word: (t >> 8) 2^-24, computed as the float of t with
// its low byte cleared (at most 24 significant bits, so the conversion is
// exact) times 2^-32.  The mask fuses with the last tempering XOR into one
// three-input logic instruction, which the shift would not.
template <int OM>
__device__ __forceinline__ uint32_t mt_conv(uint32_t t) {
  if constexpr (OM == OUT_F32) return __float_as_uint(__uint2float_rn(t & 0xFFFFFF00u) * 0x1p-32f);
  else return t;
}

// The twist's matrix constant a = 0x9908B0DF (Section 3.7), read from the
// constant bank so that its product with the low bit of y below stays a
// multiply on the FMA pipe instead of becoming a select on the integer ALU,
// which this kernel keeps busy.
__constant__ uint32_t c_mt_a = 0x9908B0DFu;

// One new word of the twist: y = the upper bit of X_k (a) over the lower 31
// bits of X_{k+1} (b), shifted right once, XOR a when y's low bit (b's) is
// set, XOR the lag word f.  Written out as four integer instructions (merge,
// shift, low bit, three-way XOR) and the multiply: left to itself the
// compiler spends one more integer instruction per word on it.
__device__ __forceinline__ uint32_t mt_mix(uint32_t a, uint32_t b, uint32_t f) {
  uint32_t r;
  asm("{\n\t"
      ".reg .b32 y, m, l;\n\t"
      "lop3.b32 y, %1, %2, 0x7FFFFFFF, 0xD8;\n\t"   // (b & 0x7FFFFFFF) | (a & 0x80000000)
      "shr.u32 y, y, 1;\n\t"
      "and.b32 l, %2, 1;\n\t"
      "mul.lo.u32 m, l, %4;\n\t"                    // a or 0
      "lop3.b32 %0, %3, y, m, 0x96;\n\t"            // f ^ y ^ m
      "}"
      : "=r"(r)
      : "r"(a), "r"(b), "r"(f), "r"(c_mt_a));
  return r;
}

// Temper the new quad v = X_k .. X_{k+3} and hand it to the output: o[k]
// onwards (16-byte stores when vec; PARTIAL: only entries k < take), or the
// fused half-sweep's sites e0 + k onwards.
template <int OM, bool PARTIAL>
__device__ __forceinline__ void mt_emit(uint4 v, int k, uint32_t* o, int take, bool vec,
                                        const FillDesc* d, uint64_t e0) {
  uint4 t;
  t.x = mt_conv<OM>(mt_temper(v.x));
  t.y = mt_conv<OM>(mt_temper(v.y));
  t.z = mt_conv<OM>(mt_temper(v.z));
  t.w = mt_conv<OM>(mt_temper(v.w));
  if constexpr (OM == OUT_ISING) {   // e0 + k: element index of word k
    if (!PARTIAL) {
      put4<OM, 32>(*d, nullptr, e0 + k, t);
    } else {
      if (k < take) put1<OM>(*d, nullptr, e0 + k, t.x);
      if (k + 1 < take) put1<OM>(*d, nullptr, e0 + k + 1, t.y);
      if (k + 2 < take) put1<OM>(*d, nullptr, e0 + k + 2, t.z);
      if (k + 3 < take) put1<OM>(*d, nullptr, e0 + k + 3, t.w);
    }
  } else if (!PARTIAL && vec) {
    st_chunk<OM, 32>(o + k, t);
  } else {
    if constexpr (OM == OUT_F64) {   // take and the table offset are even
      if (!PARTIAL || k < take) st_pair<32>(o + k, t.x, t.y);
      if (!PARTIAL || k + 2 < take) st_pair<32>(o + k + 2, t.z, t.w);
    } else {
      if (!PARTIAL || k < take) st_out(o + k, t.x);
      if (!PARTIAL || k + 1 < take) st_out(o + k + 1, t.y);
      if (!PARTIAL || k + 2 < take) st_out(o + k + 2, t.z);
      if (!PARTIAL || k + 3 < take) st_out(o + k + 3, t.w);
    }
  }
}

// Start of the four lag words of the quad at k (a multiple of 4), one word
// before them: X_{k+397} (old) for k <= 224, X_{k-227} (already new) from
// k = 228 on.  The quad at 224 takes old words 621..623 and new X_0, which
// is the word after its lag quad; both forms start on a 16-byte boundary.
__device__ __forceinline__ int mt_lag_base(int k) { return k <= 224 ? k + 396 : k - 228; }

// One twist of a stream's table (Appendix A, "Mersenne twister"), in place,
// by the LPS lanes that own the stream (32: a warp; 16: half a warp, the
// warp's other half twisting another stream in step), in chunks of
// 4 LPS QPL entries (five of 128 for both forms); lane u owns the QPL quads
// k .. k+3, k = k0 + 4 LPS q + 4 u, so each lane has QPL independent quads
// between two syncs.  Any chunk size up to 227 keeps the in-place order
// valid.  A quad needs its own four words and the next one, X_{k+4}, and
// the four lag words (mt_lag_base), which are the last three of an aligned
// 16-byte quad and the first word of the next one.  Each lane loads its own
// quad and its aligned lag quad with one 16-byte shared load each; the two
// words after them are the first words that lane u+1 loaded, passed on by a
// shuffle (the group's last lane takes lane 0's next row, and in the last
// row loads them itself).  Each new word is tempered and, if o != null,
// written to o[k] (16-byte stores when VEC); PARTIAL: only entries k < take
// are written.
template <int OM, bool PARTIAL, int LPS = 32, int QPL = 1>
__device__ __forceinline__ void mt_twist(uint32_t* s, int lane, uint32_t* o, int take, bool vec,
                                         const FillDesc* d = nullptr, uint64_t e0 = 0) {
  constexpr int CH = 4 * LPS * QPL;
  static_assert(CH <= 227, "a chunk may not reach its own lags");
#pragma unroll
  for (int k0 = 0; k0 < 624; k0 += CH) {
    uint4 a[QPL], f[QPL];
    uint32_t b[QPL];
#pragma unroll
    for (int q = 0; q < QPL; q++) {
      const int kr = k0 + 4 * LPS * q;     // first quad of the row
      const int k = kr + 4 * lane;
      a[q] = make_uint4(0, 0, 0, 0);
      f[q] = a[q];
      if (k < 624) {
        a[q] = *reinterpret_cast<const uint4*>(s + k);
        // compile-time base when the whole row is on one side of 224 / 228
        const int base = kr + 4 * LPS - 4 <= 224 ? k + 396 : (kr >= 228 ? k - 228 : mt_lag_base(k));
        f[q] = *reinterpret_cast<const uint4*>(s + base);
      }
    }
#pragma unroll
    for (int q = 0; q < QPL; q++) {
      uint32_t na = a[q].x, nf = f[q].x;
      if (q + 1 < QPL && lane == 0) {        // lane LPS-1 reads lane 0: the next row
        na = a[q + 1].x;
        nf = f[q + 1].x;
      }
      b[q] = __shfl_sync(0xFFFFFFFFu, na, (lane + 1) & (LPS - 1), LPS);
      const uint32_t h = __shfl_sync(0xFFFFFFFFu, nf, (lane + 1) & (LPS - 1), LPS);
      f[q] = make_uint4(f[q].y, f[q].z, f[q].w, h);
    }
    {
      const int kn = k0 + CH;                // the quad after the chunk (old)
      if (kn < 624 && lane == LPS - 1) {
        b[QPL - 1] = s[kn];
        f[QPL - 1].w = s[mt_lag_base(kn)];
      }
    }
#pragma unroll
    for (int q = 0; q < QPL; q++) {          // the table's last quad: X_624 is the new X_0
      const int kr = k0 + 4 * LPS * q;
      if (kr <= 620 && 620 < kr + 4 * LPS && 4 * lane + kr == 620) {
        b[q] = s[0];
        f[q].w = s[mt_lag_base(624)];
      }
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < QPL; q++) {
      const int k = k0 + 4 * LPS * q + 4 * lane;
      if (k >= 624) continue;
      uint4 v;
      v.x = mt_mix(a[q].x, a[q].y, f[q].x);
      v.y = mt_mix(a[q].y, a[q].z, f[q].y);
      v.z = mt_mix(a[q].z, a[q].w, f[q].z);
      v.w = mt_mix(a[q].w, b[q], f[q].w);
      *reinterpret_cast<uint4*>(s + k) = v;
      if (o != nullptr) mt_emit<OM, PARTIAL>(v, k, o, take, vec, d, e0);
    }
    __syncwarp();
  }
}

// Whole 624-word blocks of a fill, with each lane's own quads of the table
// held in registers from block to block (lane u owns the quads k = CH c +
// 4 LPS q + 4 u of every block, so after a twist its new quads are the old
// ones of the next block).  The table in shared memory is kept as a mirror:
// every new quad is stored there too, for the other lanes' lag reads, so
// the only shared loads of a quad are its aligned lag quad (mt_lag_base)
// and, for the group's last lane only, the two words after the row (its
// X_{k+4} and lag word); the other lanes get those from lane u+1 by a
// shuffle.  The table's last quad, whose next word is the new X_0, loads
// both too.
template <int OM, int LPS, int QPL, bool VEC>
__device__ __forceinline__ void mt_blocks_reg(uint32_t* s, int lane, uint32_t* o, uint64_t nb,
                                              const FillDesc* d, uint64_t e0) {
  constexpr int CH = 4 * LPS * QPL, NCH = (624 + CH - 1) / CH;
  static_assert(CH <= 227, "a chunk may not reach its own lags");
  static_assert((LPS & (LPS - 1)) == 0, "lane u+1 is taken modulo a power of two");
  uint4 A[NCH][QPL];
#pragma unroll
  for (int c = 0; c < NCH; c++)
#pragma unroll
    for (int q = 0; q < QPL; q++) {
      const int k = c * CH + 4 * LPS * q + 4 * lane;
      A[c][q] = k < 624 ? *reinterpret_cast<const uint4*>(s + k) : make_uint4(0, 0, 0, 0);
    }
  for (uint64_t blk = 0; blk < nb; blk++) {
    uint32_t* ob = o != nullptr ? o + blk * 624 : nullptr;
    const uint64_t eb = e0 + blk * 624;
#pragma unroll
    for (int c = 0; c < NCH; c++) {
      const int k0 = c * CH;
      uint4 F[QPL];
#pragma unroll
      for (int q = 0; q < QPL; q++) {
        const int kr = k0 + 4 * LPS * q, k = kr + 4 * lane;
        F[q] = make_uint4(0, 0, 0, 0);
        if (k < 624) {
          const int base = kr + 4 * LPS - 4 <= 224 ? k + 396 : (kr >= 228 ? k - 228 : mt_lag_base(k));
          F[q] = *reinterpret_cast<const uint4*>(s + base);
        }
      }
      uint32_t b[QPL], h[QPL];
#pragma unroll
      for (int q = 0; q < QPL; q++) {
        b[q] = __shfl_sync(0xFFFFFFFFu, A[c][q].x, (lane + 1) & (LPS - 1), LPS);
        h[q] = __shfl_sync(0xFFFFFFFFu, F[q].x, (lane + 1) & (LPS - 1), LPS);
        const int kn = k0 + 4 * LPS * (q + 1);   // the next row's first quad (old)
        if (kn < 624 && lane == LPS - 1) {       // predicated loads, no selects
          b[q] = s[kn];
          h[q] = s[mt_lag_base(kn)];
        }
      }
#pragma unroll
      for (int q = 0; q < QPL; q++) {      // X_624 is the new X_0
        const int kr = k0 + 4 * LPS * q;
        if (kr <= 620 && 620 < kr + 4 * LPS && 4 * lane + kr == 620) {
          b[q] = s[0];
          h[q] = s[mt_lag_base(624)];
        }
      }
#pragma unroll
      for (int q = 0; q < QPL; q++) {
        const int k = k0 + 4 * LPS * q + 4 * lane;
        if (k >= 624) continue;
        const uint4 a = A[c][q], f = F[q];
        uint4 v;
        v.x = mt_mix(a.x, a.y, f.y);
        v.y = mt_mix(a.y, a.z, f.z);
        v.z = mt_mix(a.z, a.w, f.w);
        v.w = mt_mix(a.w, b[q], h[q]);
        *reinterpret_cast<uint4*>(s + k) = v;
        A[c][q] = v;
        if (ob != nullptr) mt_emit<OM, false>(v, k, ob, 624, VEC, d, eb);
      }
      __syncwarp();
    }
  }
}

// Stream `row` of a fill by the LPS lanes that own it (lane u of them); s
// is its 624-word table.  With LPS = 16 the two halves of a warp run two
// streams in step: every branch that holds a __syncwarp is taken by the
// whole warp (a 624-word block is twisted as partial or unaligned if either
// stream needs it), and a half whose row is past the end (inactive) runs
// along without touching memory outside shared memory.
template <int OM, int LPS = 32, int QPL = 1, bool REG = true>
__device__ __forceinline__ void mt_stream(const FillDesc& d, uint64_t row, uint32_t* s, int lane,
                                          bool active = true) {
  uint32_t* gs = d.state + row * 624;
  if (active)
    for (int k = lane; k < 624; k += LPS) s[k] = gs[k];
  __syncwarp();

  uint32_t* out = static_cast<uint32_t*>(d.out);
  const bool store = active && out != nullptr;
  uint32_t* orow = store ? out + row * d.pitch : nullptr;
  const uint64_t n = d.n_per;
  // Draws of this row that are written (all n unless the element limit cuts
  // the row); the stream still advances by n.
  uint64_t nv = n;
  if (store && d.limit - row * d.pitch < nv) nv = d.limit - row * d.pitch;
  uint64_t j = 0;
  const uint32_t mti = d.pos;
  if (mti < 624 && n > 0) {  // rest of the current table
    const uint64_t h = (624 - mti) < n ? (624 - mti) : n;
    if (store)
      for (uint64_t k = lane; k < h && k < nv; k += LPS)
        if constexpr (OM == OUT_F64) {
          if ((k & 1) == 0) st_pair<32>(orow + k, mt_temper(s[mti + k]), mt_temper(s[mti + k + 1]));
        } else {
          put1<OM>(d, orow + k, row * d.pitch + k, mt_conv<OM>(mt_temper(s[mti + k])));
        }
    j = h;
  }
  // 16-byte output stores need the row position j to sit on a 16-byte boundary.
  bool vec = !store || ((reinterpret_cast<uintptr_t>(orow + j) & 15) == 0);
  if (LPS < 32) vec = __all_sync(0xFFFFFFFFu, vec);
  if constexpr (REG && OM != OUT_ISING) {
    // Leading blocks that are whole for both streams of the warp (or the
    // warp's one stream) run with the lanes' quads in registers
    // (mt_blocks_reg); the rest as below.  (Not in the batched kernel,
    // whose 256-thread blocks it would push into spills.)
    // (Not for the fused half-sweep: its site updates need the registers,
    // and at 96 per thread the 8,192-stream fill no longer fits one wave.)
    uint64_t nb = (n - j) / 624;
    if (store) {
      const uint64_t w = nv > j ? (nv - j) / 624 : 0;
      if (w < nb) nb = w;
    }
    const uint32_t nb32 = __reduce_min_sync(0xFFFFFFFFu, nb > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)nb);
    if (nb32 > 0) {   // vec is the same for the whole warp
      if (vec)
        mt_blocks_reg<OM, LPS, QPL, true>(s, lane, store ? orow + j : nullptr, nb32, &d, row * d.pitch + j);
      else
        mt_blocks_reg<OM, LPS, QPL, false>(s, lane, store ? orow + j : nullptr, nb32, &d, row * d.pitch + j);
      j += (uint64_t)nb32 * 624;
    }
  }
  while (n - j >= 624) {
    bool whole = !store || j + 624 <= nv;
    if (LPS < 32) whole = __all_sync(0xFFFFFFFFu, whole);
    if (whole)
      mt_twist<OM, false, LPS, QPL>(s, lane, store ? orow + j : nullptr, 624, vec, &d, row * d.pitch + j);
    else
      mt_twist<OM, true, LPS, QPL>(s, lane, store ? orow + j : nullptr,
                              (int)(store && nv > j ? (nv - j < 624 ? nv - j : 624) : 0), false, &d,
                              row * d.pitch + j);
    j += 624;
  }
  if (j < n) {
    const uint64_t take = store && nv > j ? (nv - j < n - j ? nv - j : n - j) : 0;
    mt_twist<OM, true, LPS, QPL>(s, lane, store ? orow + j : nullptr, (int)take, false, &d, row * d.pitch + j);
  }
  if (active)
    for (int k = lane; k < 624; k += LPS) gs[k] = s[k];
  __syncwarp();
}

// SPW streams per warp (1: a warp per stream; 2: a half-warp each, which
// halves the warps of a fill so that every stream of a large handle is
// resident in one wave).
template <int WPB, int OM, int SPW>
__global__ void __launch_bounds__(WPB * 32) k_fill_mt(const FillDesc d) {
  __shared__ __align__(16) uint32_t table[WPB * SPW][624];
  constexpr int LPS = 32 / SPW;
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int half = lane / LPS;
  const uint64_t row0 = ((uint64_t)blockIdx.x * WPB + wi) * SPW;
  if (row0 >= d.n_rows) return;  // whole warp leaves; no CTA-wide barriers below
  const uint64_t row = row0 + half;
  mt_stream<OM, LPS, SPW>(d, row, table[wi * SPW + half], lane % LPS, row < d.n_rows);
}

// Batched MT19937 fills: each warp pops an item (up to 2 streams of one
// request) and fills them one after the other in its own table.
template <int WPB, bool F32>
__global__ void __launch_bounds__(WPB * 32) k_batch_mt(const BatchQueue q) {
  __shared__ __align__(16) uint32_t table[WPB][624];
  __shared__ FillDesc desc[WPB];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  for (;;) {
    const uint32_t it = pop_warp(q.counter);
    if (it >= q.n_items) break;
    const BatchItem I = q.items[it];
    FillDesc& d = desc[wi];
    __syncwarp();
    load_desc(&d, q.reqs[I.req].d, lane, 32);
    __syncwarp();
    for (uint32_t k = 0; k < I.rows; k++)
      mt_stream<F32 ? OUT_F32 : OUT_U32, 32, 1, false>(d, I.row0 + k, table[wi], lane);
  }
}

// Jump-ahead (see k_mt_jump.cu): rows [r0, r1) of a table array become
// g(T) applied to row r - src_off and moved one more word on, where T moves
// a table one word along the sequence of Appendix A, "Mersenne twister".
// Word j of the result is the XOR, over the coefficients g_i = 1, of word
// 1 + i + j of the word sequence that the source table starts.  A warp
// walks that sequence 624 words at a time: the current table and the next
// (twisted from a copy) sit side by side in shared memory, so the words
// 1 + i + j of a block of 624 values of i are one contiguous window.  Lane l
// owns result words 20 l .. 20 l + 19 in registers and takes sixteen
// coefficients at a time: the 35 words they need start one word past a
// 16-byte boundary (i is a multiple of 16 and 1 + i + 20 l = 1 mod 4), so
// they are ten aligned 16-byte shared loads (lanes 80 bytes apart hit eight
// different bank quads), shared by the sixteen coefficients.  Each nibble
// of set coefficients (BITS, a compile-time variant) is folded with
// three-input XORs.
//
// The 19937 coefficients are 32 blocks of 624.  A table's blocks can be
// split over S warps (segments of ceil(32 / S) blocks): segment s first
// twists its copy of the source table forward by its first block, then
// accumulates its blocks and XORs its partial result into the (zeroed)
// destination row with atomics.  S = 1 stores the result directly and may
// run in place (destination row = source row).
template <int OFF, int BITS>
__device__ __forceinline__ void mt_poly_nib(uint32_t (&acc)[20], const uint32_t (&win)[40]) {
#pragma unroll
  for (int t = 0; t < 20; t++) {
    uint32_t x = acc[t];
    if (BITS & 1) x ^= win[OFF + 1 + t];
    if (BITS & 2) x ^= win[OFF + 2 + t];
    if (BITS & 4) x ^= win[OFF + 3 + t];
    if (BITS & 8) x ^= win[OFF + 4 + t];
    acc[t] = x;
  }
}

template <int OFF>
__device__ __forceinline__ void mt_poly_nib_any(uint32_t bits4, uint32_t (&acc)[20],
                                                const uint32_t (&win)[40]) {
  switch (bits4) {
#define PRNG_MT_NIB(b) case b: mt_poly_nib<OFF, b>(acc, win); break;
    PRNG_MT_NIB(1) PRNG_MT_NIB(2) PRNG_MT_NIB(3) PRNG_MT_NIB(4) PRNG_MT_NIB(5)
    PRNG_MT_NIB(6) PRNG_MT_NIB(7) PRNG_MT_NIB(8) PRNG_MT_NIB(9) PRNG_MT_NIB(10)
    PRNG_MT_NIB(11) PRNG_MT_NIB(12) PRNG_MT_NIB(13) PRNG_MT_NIB(14) PRNG_MT_NIB(15)
#undef PRNG_MT_NIB
    default: break;
  }
}

template <int WPB>
__global__ void __launch_bounds__(WPB * 32) k_mt_poly_apply(const __grid_constant__ MtPoly g,
                                                            uint32_t* state, uint64_t r0,
                                                            uint64_t r1, uint64_t src_off,
                                                            uint32_t S) {
  constexpr int D = 19937, NB = (D + 623) / 624;
  // current table | next table | room for lane 31's over-reach (its words
  // past 623 are computed and dropped; its last window ends at word 1267)
  __shared__ __align__(16) uint32_t buf[WPB][1280];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const uint64_t w = (uint64_t)blockIdx.x * WPB + wi;
  const uint64_t r = r0 + w / S;
  if (r >= r1) return;  // whole warp; no CTA-wide barriers below
  const int per = (NB + (int)S - 1) / (int)S;
  const int b0 = (int)(w % S) * per, b1 = b0 + per < NB ? b0 + per : NB;
  if (b0 >= b1) return;
  uint32_t* B = buf[wi];
  const uint32_t* src = state + (r - src_off) * 624;
  for (int k = lane; k < 624; k += 32) B[k] = src[k];
  for (int k = 1248 + lane; k < 1280; k += 32) B[k] = 0;
  for (int b = 0; b < b0; b++) {   // to the segment's first block
    __syncwarp();
    mt_twist<OUT_U32, false>(B, lane, nullptr, 624, false);
  }
  uint32_t acc[20];
#pragma unroll
  for (int t = 0; t < 20; t++) acc[t] = 0;
  for (int i0 = b0 * 624; i0 < b1 * 624 && i0 < D; i0 += 624) {
    __syncwarp();
    for (int k = lane; k < 624; k += 32) B[624 + k] = B[k];
    __syncwarp();
    mt_twist<OUT_U32, false>(B + 624, lane, nullptr, 624, false);  // the next 624 words
    const int i1 = i0 + 624 < D ? i0 + 624 : D;
    for (int i = i0; i < i1; i += 16) {   // i0 and i are multiples of 16: half of one word
      uint32_t bits = (g.w[i >> 5] >> (i & 31)) & 0xFFFFu;
      if (i1 - i < 16) bits &= (1u << (i1 - i)) - 1u;
      if (!bits) continue;
      const int a = (i - i0) + 20 * lane;          // 16-byte aligned; the window starts at a + 1
      uint32_t win[40];
#pragma unroll
      for (int q = 0; q < 10; q++) {
        const uint4 v = *reinterpret_cast<const uint4*>(B + a + 4 * q);
        win[4 * q] = v.x; win[4 * q + 1] = v.y; win[4 * q + 2] = v.z; win[4 * q + 3] = v.w;
      }
      mt_poly_nib_any<0>(bits & 0xFu, acc, win);
      mt_poly_nib_any<4>((bits >> 4) & 0xFu, acc, win);
      mt_poly_nib_any<8>((bits >> 8) & 0xFu, acc, win);
      mt_poly_nib_any<12>(bits >> 12, acc, win);
    }
    __syncwarp();
    for (int k = lane; k < 624; k += 32) B[k] = B[624 + k];
  }
  uint32_t* dst = state + r * 624;
  if (S == 1) {
#pragma unroll
    for (int t = 0; t < 20; t++)
      if (20 * lane + t < 624) dst[20 * lane + t] = acc[t];
  } else {
#pragma unroll
    for (int t = 0; t < 20; t++)
      if (20 * lane + t < 624) atomicXor(dst + 20 * lane + t, acc[t]);
  }
}

cudaError_t launch_mt_poly_apply(const MtPoly& g, uint32_t* state, uint64_t r0, uint64_t r1,
                                 uint64_t src_off, cudaStream_t s) {
  if (r1 <= r0) return cudaSuccess;
  constexpr int WPB = 4;
  // Few tables: split each table's coefficient blocks over up to 32 warps
  // (destination rows zeroed first), so that a pass keeps about 4096 warps
  // busy.  In place (src_off = 0) needs the unsplit form.
  const uint64_t tables = r1 - r0;
  uint32_t S = 1;
  if (src_off != 0)
    while (S < 32 && tables * S < 4096) S *= 2;
  if (S > 1) {
    const cudaError_t e = cudaMemsetAsync(state + r0 * 624, 0, tables * 624 * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
  }
  const uint64_t blocks = (tables * S + WPB - 1) / WPB;
  if (blocks > 0x7FFFFFFFull) return cudaErrorInvalidValue;
  k_mt_poly_apply<WPB><<<(unsigned)blocks, WPB * 32, 0, s>>>(g, state, r0, r1, src_off, S);
  return cudaGetLastError();
}

cudaError_t launch_batch_mt(const BatchQueue& q, Tile t, bool f32, cudaStream_t s) {
  (void)t;
  if (q.n_items == 0) return cudaSuccess;
  const uint32_t cap = (uint32_t)sm_count() * (2048 / 256);
  const uint32_t need = (q.n_items + 7) / 8;
  const uint32_t grid = need < cap ? need : cap;
  if (f32) k_batch_mt<8, true><<<grid, 256, 0, s>>>(q);
  else k_batch_mt<8, false><<<grid, 256, 0, s>>>(q);
  return cudaGetLastError();
}

template <int WPB, int OM, int SPW>
static cudaError_t launch_mt(const FillDesc& d, cudaStream_t s) {
  const uint64_t grid = (d.n_rows + WPB * SPW - 1) / (WPB * SPW);
  k_fill_mt<WPB, OM, SPW><<<(unsigned)grid, WPB * 32, 0, s>>>(d);
  return cudaGetLastError();
}

// Tile: threads per CTA (64, 128, 256; 32 with two streams per warp, so that
// the CTAs of a large fill spread evenly over the SMs) and, in `stages`,
// streams per warp.
cudaError_t launch_fill_mt(const FillDesc& d, Tile t, cudaStream_t s) {
  if (d.n_rows == 0 || d.n_per == 0) return cudaSuccess;
  return with_mode(d.mode, [&](auto m) {
    constexpr int OM = decltype(m)::value;
    if (t.stages == 2) {
      if (t.threads == 32) return launch_mt<1, OM, 2>(d, s);
      if (t.threads == 64) return launch_mt<2, OM, 2>(d, s);
      if (t.threads == 256) return launch_mt<8, OM, 2>(d, s);
      return launch_mt<4, OM, 2>(d, s);
    }
    if (t.threads == 64) return launch_mt<2, OM, 1>(d, s);
    if (t.threads == 256) return launch_mt<8, OM, 1>(d, s);
    return launch_mt<4, OM, 1>(d, s);
  });
}

}  // namespace prng
