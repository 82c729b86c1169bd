// k_ranlux_p97.cu -- RANLUX kernels and launchers for luxury p = 97.
#include "ranlux.cuh"

namespace prng {
PRNG_RANLUX_LEVEL(97)
}  // namespace prng
