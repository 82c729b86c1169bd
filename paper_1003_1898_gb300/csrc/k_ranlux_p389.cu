// k_ranlux_p389.cu -- RANLUX kernels and launchers for luxury p = 389.
#include "ranlux.cuh"

namespace prng {
PRNG_RANLUX_LEVEL(389)
}  // namespace prng
