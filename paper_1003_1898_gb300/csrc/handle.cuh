// handle.cuh -- the handle behind the opaque prng_state and the host-side
// bookkeeping shared by the single-handle and batched entry points.
#pragma once

#include <cstdint>

#include "common.cuh"

struct prng_state {
  int gen;
  int p;                 // RANLUX luxury p (0 for the others)
  uint64_t n_streams;
  uint32_t* d_state;     // device state, layout in common.cuh
  uint32_t pos;          // RANLUX: draws delivered from the open block; MT: mti
  int device;
};

namespace prng {

// Luxury level or p -> p: levels 0..4 are the standard p = 24, 48, 97, 223,
// 389 (Appendix A, "RANLUX"); p itself is accepted, and so are the planar
// scheme's p = 120, 240, 408 (Section 3.6: 96, 216, 384 discarded after each
// 24 delivered; its level 1, p = 48, is standard p = 48).
inline int luxury_to_p(uint32_t luxury) {
  static const int P[8] = {24, 48, 97, 223, 389, 120, 240, 408};
  if (luxury <= 4) return P[luxury];
  for (int i = 0; i < 8; i++)
    if ((int)luxury == P[i]) return P[i];
  return -1;
}

inline uint32_t initial_pos(int gen) { return gen == MT19937 ? 624u : 0u; }

// Position after n more draws (all streams of a handle move together).
inline uint32_t advance_pos(int gen, uint32_t pos, uint64_t n) {
  if (n == 0) return pos;
  if (gen == RANLUX) {
    const uint64_t h = pos < 24 ? (24 - pos < n ? 24 - pos : n) : 0;
    const uint64_t r = n - h;
    return r == 0 ? (uint32_t)(pos + h) : (uint32_t)((r - 1) % 24 + 1);
  }
  if (gen == MT19937) {
    const uint64_t h = pos < 624 ? (624 - pos < n ? 624 - pos : n) : 0;
    const uint64_t r = n - h;
    return r == 0 ? (uint32_t)(pos + h) : (uint32_t)((r - 1) % 624 + 1);
  }
  return 0;
}

}  // namespace prng
