// k_ranlux_p223.cu -- RANLUX kernels and launchers for luxury p = 223.
#include "ranlux.cuh"

namespace prng {
PRNG_RANLUX_LEVEL(223)
}  // namespace prng
