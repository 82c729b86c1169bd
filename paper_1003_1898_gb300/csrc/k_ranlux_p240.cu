// k_ranlux_p240.cu -- RANLUX kernels and launchers for luxury p = 240 (the
// planar scheme of Section 3.6: 24 delivered, 216 discarded).
#include "ranlux.cuh"

namespace prng {
PRNG_RANLUX_LEVEL(240)
}  // namespace prng
