// k_ranlux_p24.cu -- RANLUX kernels and launchers for luxury p = 24.
#include "ranlux.cuh"

namespace prng {
PRNG_RANLUX_LEVEL(24)
}  // namespace prng
