// scratch.cuh -- stream-ordered scratch for the jump fills' chunk-start
// tables, from a memory pool the library creates once per device and that
// keeps its memory for reuse (the device's default pool would hand freed
// memory back at every synchronisation, so that each call allocated afresh).
#pragma once

#include <cstddef>
#include <cuda_runtime.h>

namespace prng {

cudaError_t scratch_alloc(void** p, size_t bytes, cudaStream_t s);
cudaError_t scratch_free(void* p, cudaStream_t s);

}  // namespace prng
