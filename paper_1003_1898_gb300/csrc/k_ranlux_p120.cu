// k_ranlux_p120.cu -- RANLUX kernels and launchers for luxury p = 120 (the
// planar scheme of Section 3.6: 24 delivered, 96 discarded).
#include "ranlux.cuh"

namespace prng {
PRNG_RANLUX_LEVEL(120)
}  // namespace prng
