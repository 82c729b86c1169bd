// k_ranlux_p408.cu -- RANLUX kernels and launchers for luxury p = 408 (the
// planar scheme of Section 3.6: 24 delivered, 384 discarded).
#include "ranlux.cuh"

namespace prng {
PRNG_RANLUX_LEVEL(408)
}  // namespace prng
