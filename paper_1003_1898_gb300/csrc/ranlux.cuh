// ranlux.cuh -- RANLUX fill and skip kernels (Section 3.6; Appendix A, "AWC and SWB"
// and "RANLUX"), instantiated once per luxury level in k_ranlux_p<P>.cu.
//
// One thread per stream.  In the hot loop the 24-word RCARRY ring and the
// borrow live in registers and the ring is walked 24 steps at a time with a
// compile-time phase, so both lags (x_{n-10}, x_{n-24}) are fixed registers
// and no register is indexed at run time; 24 steps at a time run as one
// subtract-with-borrow chain (swb24).  A luxury cycle is 24 delivered
// steps plus p - 24 discarded ones; p - 24 = 24 q + r runs as q 24-step
// chains, one r-step chain and one fixed register permutation.
//
// The pieces whose length is only known at run time -- the head of a fill
// that resumes inside a block and the tail of a fill that stops inside one --
// run on a copy of the ring in shared memory with run-time indices (a few
// dozen steps per call), and the registers are loaded from / stored to that
// copy with the matching rotation.
//
// Delivered draws are staged in a row-major shared tile with 16-byte stores
// and written out 16 bytes at a time (RowFlusher), so the stream-major HBM
// writes are contiguous runs of each row.
#pragma once

#include "batch.cuh"

namespace prng {

// In registers each word is held as X = x * 2^8 (the 24-bit value in the
// high bits, low byte 0).  Then one 32-bit subtract-with-borrow computes an
// SWB step exactly: X10 - X24 - c has x10 - x24 - c (mod 2^24) in its high
// 24 bits, and it borrows out of bit 31 exactly when x10 - x24 - c < 0,
// because the low bytes of both operands are 0.  Only the low byte needs
// clearing (it becomes 0xFF when c = 1).

// One SWB step at compile-time ring phase k: V[j] = R[(j + k) % 24],
// x_n = (x_{n-10} - x_{n-24} - c) mod 2^24, c = borrow.
__device__ __forceinline__ void swb_step(uint32_t (&R)[24], uint32_t& c, const int k) {
  const int i0 = k % 24, i14 = (k + 14) % 24;
  const uint32_t a = R[i14];
  const uint32_t t = a - R[i0] - c;
  c = t > a ? 1u : 0u;          // borrow: R[i0] + c > a (no overflow, low bytes are 0)
  R[i0] = t & 0xFFFFFF00u;
}

// One SWB step of a carry chain on asm operands k (the word replaced) and
// l (its lag-10 partner): X_k = X_l - X_k - borrow, low byte cleared.
#define LUX_SWB(k, l) "subc.cc.u32 %" k ", %" l ", %" k ";\n\tand.b32 %" k ", %" k ", -256;\n\t"

// 24 steps from phase 0 as one subtract-with-borrow chain: the borrow
// travels in the carry flag, so the serial dependence per step is a single
// instruction, and it enters and leaves the flag once per 24 steps.  Step k
// replaces word k with word (k + 14) % 24 minus word k; for k >= 10 that
// partner was already replaced earlier in the chain, as the recurrence
// requires.  The ring returns to phase 0.
__device__ __forceinline__ void swb24(uint32_t (&R)[24], uint32_t& c) {
  asm("{\n\t"
      ".reg .u32 t;\n\t"
      "sub.cc.u32 t, 0, %24;\n\t"
      LUX_SWB("0", "14")
      LUX_SWB("1", "15")
      LUX_SWB("2", "16")
      LUX_SWB("3", "17")
      LUX_SWB("4", "18")
      LUX_SWB("5", "19")
      LUX_SWB("6", "20")
      LUX_SWB("7", "21")
      LUX_SWB("8", "22")
      LUX_SWB("9", "23")
      LUX_SWB("10", "0")
      LUX_SWB("11", "1")
      LUX_SWB("12", "2")
      LUX_SWB("13", "3")
      LUX_SWB("14", "4")
      LUX_SWB("15", "5")
      LUX_SWB("16", "6")
      LUX_SWB("17", "7")
      LUX_SWB("18", "8")
      LUX_SWB("19", "9")
      LUX_SWB("20", "10")
      LUX_SWB("21", "11")
      LUX_SWB("22", "12")
      LUX_SWB("23", "13")
      "subc.u32 %24, 0, 0;\n\t"
      "and.b32 %24, %24, 1;\n\t"
      "}"
      : "+r"(R[0]), "+r"(R[1]), "+r"(R[2]), "+r"(R[3]), "+r"(R[4]), "+r"(R[5]), "+r"(R[6]),
        "+r"(R[7]), "+r"(R[8]), "+r"(R[9]), "+r"(R[10]), "+r"(R[11]), "+r"(R[12]), "+r"(R[13]),
        "+r"(R[14]), "+r"(R[15]), "+r"(R[16]), "+r"(R[17]), "+r"(R[18]), "+r"(R[19]),
        "+r"(R[20]), "+r"(R[21]), "+r"(R[22]), "+r"(R[23]), "+r"(c));
}

// The first N steps from phase 0 (N <= 10, so every partner, word 14 + k,
// is still unreplaced) as one chain; lengths without a chain fall back to
// single steps.
template <int N>
__device__ __forceinline__ void swb_head(uint32_t (&R)[24], uint32_t& c) {
  if constexpr (N == 1) {
    asm("{\n\t"
        ".reg .u32 t;\n\t"
        "sub.cc.u32 t, 0, %1;\n\t"
        LUX_SWB("0", "2")
        "subc.u32 %1, 0, 0;\n\t"
        "and.b32 %1, %1, 1;\n\t"
        "}"
        : "+r"(R[0]), "+r"(c)
        : "r"(R[14]));
  } else if constexpr (N == 5) {
    asm("{\n\t"
        ".reg .u32 t;\n\t"
        "sub.cc.u32 t, 0, %5;\n\t"
        LUX_SWB("0", "6")
        LUX_SWB("1", "7")
        LUX_SWB("2", "8")
        LUX_SWB("3", "9")
        LUX_SWB("4", "10")
        "subc.u32 %5, 0, 0;\n\t"
        "and.b32 %5, %5, 1;\n\t"
        "}"
        : "+r"(R[0]), "+r"(R[1]), "+r"(R[2]), "+r"(R[3]), "+r"(R[4]), "+r"(c)
        : "r"(R[14]), "r"(R[15]), "r"(R[16]), "r"(R[17]), "r"(R[18]));
  } else if constexpr (N == 7) {
    asm("{\n\t"
        ".reg .u32 t;\n\t"
        "sub.cc.u32 t, 0, %7;\n\t"
        LUX_SWB("0", "8")
        LUX_SWB("1", "9")
        LUX_SWB("2", "10")
        LUX_SWB("3", "11")
        LUX_SWB("4", "12")
        LUX_SWB("5", "13")
        LUX_SWB("6", "14")
        "subc.u32 %7, 0, 0;\n\t"
        "and.b32 %7, %7, 1;\n\t"
        "}"
        : "+r"(R[0]), "+r"(R[1]), "+r"(R[2]), "+r"(R[3]), "+r"(R[4]), "+r"(R[5]), "+r"(R[6]), "+r"(c)
        : "r"(R[14]), "r"(R[15]), "r"(R[16]), "r"(R[17]), "r"(R[18]), "r"(R[19]), "r"(R[20]));
  } else {
#pragma unroll
    for (int k = 0; k < N; k++) swb_step(R, c, k);
  }
}

// new R[j] = R[(j + s) % 24] for a compile-time s.
__device__ __forceinline__ void rotate_fixed(uint32_t (&R)[24], const int s) {
  uint32_t tmp[24];
#pragma unroll
  for (int j = 0; j < 24; j++) tmp[j] = R[(j + s) % 24];
#pragma unroll
  for (int j = 0; j < 24; j++) R[j] = tmp[j];
}

// Output of a word held as X = x * 2^8: x itself, or x * 2^-24 = X * 2^-32
// (X has at most 24 significant bits, so the conversion is exact).
template <int OM>
__device__ __forceinline__ uint32_t lux_out(uint32_t X) {
  if constexpr (OM == OUT_F32) return __float_as_uint(__uint2float_rn(X) * 0x1p-32f);
  else return X >> 8;
}

template <int OM>
__device__ __forceinline__ uint32_t lux_conv(uint32_t x) {
  if constexpr (OM == OUT_F32) return __float_as_uint(__uint2float_rn(x) * 0x1p-24f);
  else return x;
}

// p - 24 discarded steps from phase 0; leaves the ring at phase 0.
template <int P>
__device__ __forceinline__ void discard_cycle(uint32_t (&R)[24], uint32_t& c) {
  constexpr int D = P - 24, Q = D / 24, RR = D % 24;
#pragma unroll
  for (int g = 0; g < Q; g++) swb24(R, c);
  swb_head<RR>(R, c);
  if constexpr (RR != 0) rotate_fixed(R, RR);
}

// `cnt` SWB steps on a ring held in shared memory (ring[j], phase `ph`),
// emitting each new word to out[k] when emit is set.
template <int OM>
__device__ __forceinline__ int swb_smem(uint32_t* ring, int ph, uint32_t& c, int cnt,
                                        uint32_t* out, bool emit) {
  for (int k = 0; k < cnt; k++) {
    const int i14 = ph + 14 < 24 ? ph + 14 : ph - 10;
    const int32_t t = (int32_t)ring[i14] - (int32_t)ring[ph] - (int32_t)c;
    c = (uint32_t)t >> 31;
    const uint32_t x = (uint32_t)t & 0xFFFFFFu;
    ring[ph] = x;
    if (emit) out[k] = lux_conv<OM>(x);
    ph = ph + 1 < 24 ? ph + 1 : 0;
  }
  return ph;
}

// Streams [row0, row0 + T) of a fill, one per thread; smem holds a
// row-major tile of T rows x SPW words (KT staged columns each).
template <int T, int KT, int P, int OM, bool LIMITED>
__device__ __forceinline__ void ranlux_rows(const FillDesc& d, uint64_t row0, uint32_t* smem) {
  static_assert(KT % 24 == 0 && KT >= 48,
                "the tile holds whole blocks; columns 24..47 double as the scratch ring");
  constexpr int SPW = KT + 4;
  const int tid = threadIdx.x;
  const uint64_t row = row0 + tid;
  const bool active = row < d.n_rows;
  const uint64_t nr = d.n_rows;
  uint32_t* out = static_cast<uint32_t*>(d.out);
  const bool store = out != nullptr;
  RowFlusher<T, SPW, LIMITED, OM, 24> fl;
  fl.init(smem, out, d.pitch, row0, nr, d.limit, &d);
  uint32_t* my = smem + tid * SPW;            // this thread's tile row
  uint32_t* ring = my + 24;                   // scratch ring in columns 24..47

  const uint64_t n = d.n_per;
  const int pos0 = (int)d.pos;
  int fill = 0;
  uint64_t g0 = 0, j = 0;
  uint32_t R[24];
  uint32_t c = 0;

  auto flush = [&]() {
    __syncthreads();
    if (store) fl.flush(g0, fill);
    __syncthreads();
    g0 += fill;
    fill = 0;
  };

  if (pos0 < 24) {
    // Finish the block a previous call left open: h draws on the shared copy.
    const int h = (int)((uint64_t)(24 - pos0) < n ? (uint64_t)(24 - pos0) : n);
    for (int jj = 0; jj < 24; jj++) ring[jj] = active ? d.state[jj * nr + row] : 0u;
    c = active ? d.state[24 * nr + row] : 0u;
    const int ph = swb_smem<OM>(ring, 0, c, h, my, store);
    fill = h;
    j = h;
    if (j == n) {  // the fill ends inside the open block
      if (active) {
        for (int jj = 0; jj < 24; jj++) {
          const int src = jj + ph < 24 ? jj + ph : jj + ph - 24;
          d.state[(uint64_t)jj * nr + row] = ring[src];
        }
        d.state[24 * nr + row] = c;
      }
      flush();
      return;
    }
#pragma unroll
    for (int jj = 0; jj < 24; jj++) R[jj] = ring[(jj + h) % 24] << 8;  // h == 24 - pos0 here
    // Flushes then come every 48 columns; they keep 64-byte-aligned row
    // runs when the first one ends on a multiple of 16 columns.  So the head
    // is flushed alone when h is a multiple of 16, and otherwise, when h = 8
    // or 24, kept in the tile with the first block written after it (h is a
    // multiple of 4, so the block's 16-byte shared stores stay aligned).
    if (!((h & 3) == 0 && ((h + 24) & 15) == 0)) flush();
  } else {
#pragma unroll
    for (int jj = 0; jj < 24; jj++) R[jj] = active ? d.state[jj * nr + row] << 8 : 0u;
    c = active ? d.state[24 * nr + row] : 0u;
  }

  // Whole blocks: discard p - 24, deliver 24, all in registers; each block
  // is six 16-byte shared stores at tile column 0 or 24 (or right after a
  // head of 8 or 24 kept in the tile).
  while (n - j >= 24) {
    discard_cycle<P>(R, c);
    if (fill + 24 > KT) flush();
    swb24(R, c);
    if (store) {
      uint4* dst = reinterpret_cast<uint4*>(my + fill);
#pragma unroll
      for (int q = 0; q < 6; q++)
        dst[q] = make_uint4(lux_out<OM>(R[4 * q]), lux_out<OM>(R[4 * q + 1]),
                            lux_out<OM>(R[4 * q + 2]), lux_out<OM>(R[4 * q + 3]));
    }
    fill += 24;
    j += 24;
  }

  if (j < n) {
    // Tail: the discard in registers, then m < 24 draws on the shared copy.
    const int m = (int)(n - j);
    discard_cycle<P>(R, c);
    if (fill > 0) flush();
#pragma unroll
    for (int jj = 0; jj < 24; jj++) ring[jj] = R[jj] >> 8;
    const int ph = swb_smem<OM>(ring, 0, c, m, my, store);
    fill = m;
    if (active) {
      for (int jj = 0; jj < 24; jj++) {
        const int src = jj + ph < 24 ? jj + ph : jj + ph - 24;
        d.state[(uint64_t)jj * nr + row] = ring[src];
      }
      d.state[24 * nr + row] = c;
    }
    flush();
    return;
  }

  if (fill > 0) flush();
  if (active) {
#pragma unroll
    for (int jj = 0; jj < 24; jj++) d.state[jj * nr + row] = R[jj] >> 8;
    d.state[24 * nr + row] = c;
  }
}

// The same fill with a per-row ring instead of a flushed tile: each
// thread's delivered blocks go to a ring of 56 words (14 16-byte chunks) in
// its shared row, and its warp writes the warp's 32 rows out 32 words (one
// aligned 128-byte line per row, when the row pitch is a multiple of 32
// words) at a time, as soon as 32 are pending.  The ring never holds more
// than 31 + 24 words, the warp's rows share one schedule (same length and
// start position), so the copy-out is a warp-level step with no CTA
// barrier.  Used for u32/f32 plain fills whose copies are 16-byte aligned:
// pitch a multiple of 4 and a start that leaves a multiple of 4 draws in
// the open block.
template <int T, int P, int OM>
__device__ __forceinline__ void ranlux_rows_ring(const FillDesc& d, uint64_t row0, uint32_t* smem) {
  constexpr int RC = 14, SPW = 4 * RC + 4;    // ring chunks; row pitch 15 chunks (odd: no conflicts)
  static_assert(T % 32 == 0, "whole warps");
  const int tid = threadIdx.x, lane = tid & 31, wi = tid >> 5;
  const uint64_t row = row0 + tid;
  const uint64_t nr = d.n_rows;
  const bool active = row < nr;
  uint32_t* out = static_cast<uint32_t*>(d.out);
  const bool store = out != nullptr;
  uint32_t* my = smem + tid * SPW;
  const uint32_t* wrows = smem + (wi * 32) * SPW;   // the warp's 32 ring rows
  const uint64_t wrow0 = row0 + (uint64_t)wi * 32;
  const int fq = lane & 7, fr = lane >> 3;         // copy-out role: chunk fq of rows fr + 4 i

  const uint64_t n = d.n_per;
  const int pos0 = (int)d.pos;
  uint64_t j = 0, fpos = 0;   // draws made / written out in this call
  int wc = 0, fc = 0;         // ring chunk of the next block / of the next copy-out
  int pend = 0;               // words in the ring not yet written out
  uint32_t R[24];
  uint32_t c = 0;

  // k chunks (4 k words, k <= 8) of every row of the warp from ring chunk fc
  // to row column fpos.
  auto copy_out = [&](int k) {
    __syncwarp();
    if (store && fq < k) {
      int ch = fc + fq;
      if (ch >= RC) ch -= RC;
#pragma unroll
      for (int i = 0; i < 8; i++) {
        const uint64_t rr = wrow0 + fr + 4 * i;
        if (rr < nr)
          st_chunk<OM, 24>(out + rr * d.pitch + fpos + 4 * fq,
                           *reinterpret_cast<const uint4*>(wrows + (fr + 4 * i) * SPW + 4 * ch));
      }
    }
    __syncwarp();
    fpos += 4 * k;
    fc += k;
    if (fc >= RC) fc -= RC;
    pend -= 4 * k;
  };

  if (pos0 < 24) {
    // Finish the open block on a shared copy of the ring (words 32..55 of
    // the row), writing its h draws to ring words 0..h-1.
    uint32_t* sring = my + 32;
    const int h = (int)((uint64_t)(24 - pos0) < n ? (uint64_t)(24 - pos0) : n);
    for (int jj = 0; jj < 24; jj++) sring[jj] = active ? d.state[jj * nr + row] : 0u;
    c = active ? d.state[24 * nr + row] : 0u;
    const int ph = swb_smem<OM>(sring, 0, c, h, my, true);
    j = h;
    if (j == n) {   // the fill ends inside the open block
      if (active) {
        for (int jj = 0; jj < 24; jj++) {
          const int src = jj + ph < 24 ? jj + ph : jj + ph - 24;
          d.state[(uint64_t)jj * nr + row] = sring[src];
        }
        d.state[24 * nr + row] = c;
        if (store)
          for (int k = 0; k < h; k++) st_out(out + row * d.pitch + k, my[k]);
      }
      return;
    }
#pragma unroll
    for (int jj = 0; jj < 24; jj++) R[jj] = sring[(jj + h) % 24] << 8;
    pend = h;          // a multiple of 4
    wc = h / 4;
  } else {
#pragma unroll
    for (int jj = 0; jj < 24; jj++) R[jj] = active ? d.state[jj * nr + row] << 8 : 0u;
    c = active ? d.state[24 * nr + row] : 0u;
  }

  while (n - j >= 24) {
    discard_cycle<P>(R, c);
    swb24(R, c);
#pragma unroll
    for (int q = 0; q < 6; q++) {
      int ch = wc + q;
      if (ch >= RC) ch -= RC;
      *reinterpret_cast<uint4*>(my + 4 * ch) =
          make_uint4(lux_out<OM>(R[4 * q]), lux_out<OM>(R[4 * q + 1]), lux_out<OM>(R[4 * q + 2]),
                     lux_out<OM>(R[4 * q + 3]));
    }
    wc += 6;
    if (wc >= RC) wc -= RC;
    pend += 24;
    j += 24;
    if (pend >= 32) copy_out(8);
  }
  if (pend > 0) copy_out(pend / 4);

  if (j < n) {
    // Tail: the discard in registers, then m < 24 draws on a shared copy
    // (row words 0..23; the draws at 24..), stored by each thread.
    const int m = (int)(n - j);
    discard_cycle<P>(R, c);
    __syncwarp();
#pragma unroll
    for (int jj = 0; jj < 24; jj++) my[jj] = R[jj] >> 8;
    const int ph = swb_smem<OM>(my, 0, c, m, my + 24, true);
    if (active) {
      if (store)
        for (int k = 0; k < m; k++) st_out(out + row * d.pitch + fpos + k, my[24 + k]);
      for (int jj = 0; jj < 24; jj++) {
        const int src = jj + ph < 24 ? jj + ph : jj + ph - 24;
        d.state[(uint64_t)jj * nr + row] = my[src];
      }
      d.state[24 * nr + row] = c;
    }
    return;
  }

  if (active) {
#pragma unroll
    for (int jj = 0; jj < 24; jj++) d.state[jj * nr + row] = R[jj] >> 8;
    d.state[24 * nr + row] = c;
  }
}

template <int T, int P, int OM>
__global__ void __launch_bounds__(T, 896 / T) k_fill_ranlux_ring(const FillDesc d) {
  extern __shared__ __align__(16) uint32_t smem[];
  ranlux_rows_ring<T, P, OM>(d, (uint64_t)blockIdx.x * T, smem);
}

template <int T, int KT, int P, int OM>
__global__ void __launch_bounds__(T, 896 / T) k_fill_ranlux(const FillDesc d) {
  extern __shared__ uint32_t smem[];
  ranlux_rows<T, KT, P, OM, false>(d, (uint64_t)blockIdx.x * T, smem);
}

// Batched RANLUX fills of luxury P: a block pops an item (T streams).
template <int T, int KT, int P, bool F32>
__global__ void __launch_bounds__(T, 768 / T) k_batch_ranlux(const BatchQueue q) {
  extern __shared__ uint32_t smem[];
  __shared__ uint32_t slot;
  for (;;) {
    const uint32_t it = pop_cta(q.counter, &slot);
    if (it >= q.n_items) break;
    const BatchItem si = q.items[it];
    __shared__ FillDesc sd;
    load_desc(&sd, q.reqs[si.req].d, threadIdx.x, T);
    __syncthreads();
    ranlux_rows<T, KT, P, F32 ? OUT_F32 : OUT_U32, true>(sd, si.row0, smem);
  }
}

template <int T, int KT, int P, bool F32>
static cudaError_t launch_bl(const BatchQueue& q, cudaStream_t s) {
  constexpr size_t bytes = (size_t)T * (KT + 4) * sizeof(uint32_t);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_batch_ranlux<T, KT, P, F32>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_ranlux<T, KT, P, F32>, T, bytes);
  const uint32_t cap = (uint32_t)sm_count() * (per_sm > 0 ? per_sm : 1);
  k_batch_ranlux<T, KT, P, F32><<<q.n_items < cap ? q.n_items : cap, T, bytes, s>>>(q);
  return cudaGetLastError();
}

template <int T, int KT, int P, int OM>
static cudaError_t launch_l(const FillDesc& d, cudaStream_t s) {
  constexpr size_t bytes = (size_t)T * (KT + 4) * sizeof(uint32_t);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_fill_ranlux<T, KT, P, OM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const uint64_t grid = (d.n_rows + T - 1) / T;
  k_fill_ranlux<T, KT, P, OM><<<(unsigned)grid, T, bytes, s>>>(d);
  return cudaGetLastError();
}

// Whether a plain fill can take the ring form: u32 or f32, every 16-byte
// copy aligned (output, pitch, and the draws left in the open block).
inline bool ranlux_ring_ok(const FillDesc& d) {
  if (d.mode != OUT_U32 && d.mode != OUT_F32) return false;
  if (d.pos < 24 && (d.pos & 3) != 0) return false;
  return d.out == nullptr || (((reinterpret_cast<uintptr_t>(d.out) & 15) == 0) && (d.pitch & 3) == 0);
}

template <int T, int P, int OM>
static cudaError_t launch_ring(const FillDesc& d, cudaStream_t s) {
  constexpr size_t bytes = (size_t)T * 60 * sizeof(uint32_t);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_fill_ranlux_ring<T, P, OM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_fill_ranlux_ring<T, P, OM>,
                               cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const uint64_t grid = (d.n_rows + T - 1) / T;
  k_fill_ranlux_ring<T, P, OM><<<(unsigned)grid, T, bytes, s>>>(d);
  return cudaGetLastError();
}

// Launchers of one luxury P for every compiled tile (defined once per P, in
// k_ranlux_p<P>.cu, so that the luxury levels compile in parallel).
template <int P>
cudaError_t ranlux_fill_p(const FillDesc& d, Tile t, cudaStream_t s) {
  const bool ring = t.cols == 56 && ranlux_ring_ok(d);
  return with_mode(d.mode, [&](auto m) {
    constexpr int OM = decltype(m)::value;
    if constexpr (OM == OUT_U32 || OM == OUT_F32) {
      if (ring) {   // cols = 56: the per-row ring with warp-level 128-byte copy-outs
        if (t.threads == 64) return launch_ring<64, P, OM>(d, s);
        if (t.threads == 256) return launch_ring<256, P, OM>(d, s);
        return launch_ring<128, P, OM>(d, s);
      }
    }
    if constexpr (P >= 97) {   // fewer flushes where the chains, not the stores, set the pace
      if (t.threads == 64 && t.cols == 96) return launch_l<64, 96, P, OM>(d, s);
    }
    if (t.threads == 64) return launch_l<64, 48, P, OM>(d, s);
    if (t.threads == 256) return launch_l<256, 48, P, OM>(d, s);
    return launch_l<128, 48, P, OM>(d, s);
  });
}

template <int P>
cudaError_t ranlux_batch_p(const BatchQueue& q, Tile t, bool f32, cudaStream_t s) {
  if (t.threads == 32) return f32 ? launch_bl<32, 48, P, true>(q, s) : launch_bl<32, 48, P, false>(q, s);
  if (t.threads == 64) return f32 ? launch_bl<64, 48, P, true>(q, s) : launch_bl<64, 48, P, false>(q, s);
  return f32 ? launch_bl<128, 48, P, true>(q, s) : launch_bl<128, 48, P, false>(q, s);
}

#define PRNG_RANLUX_LEVEL(P)                                                          \
  template cudaError_t ranlux_fill_p<P>(const FillDesc&, Tile, cudaStream_t);          \
  template cudaError_t ranlux_batch_p<P>(const BatchQueue&, Tile, bool, cudaStream_t);

#define PRNG_RANLUX_DECLARE(P)                                                               \
  extern template cudaError_t ranlux_fill_p<P>(const FillDesc&, Tile, cudaStream_t);          \
  extern template cudaError_t ranlux_batch_p<P>(const BatchQueue&, Tile, bool, cudaStream_t);

}  // namespace prng
