// k_ranlux_p48.cu -- RANLUX kernels and launchers for luxury p = 48.
#include "ranlux.cuh"

namespace prng {
PRNG_RANLUX_LEVEL(48)
}  // namespace prng
