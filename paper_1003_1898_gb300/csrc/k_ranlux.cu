// k_ranlux.cu -- RANLUX entry points (Section 3.6; Appendix A, "RANLUX"):
// dispatch on the luxury p to the launchers compiled per level (the standard
// p = 24, 48, 97, 223, 389 and the planar scheme's p = 120, 240, 408).
#include "ranlux.cuh"

namespace prng {

PRNG_RANLUX_DECLARE(24)
PRNG_RANLUX_DECLARE(48)
PRNG_RANLUX_DECLARE(97)
PRNG_RANLUX_DECLARE(223)
PRNG_RANLUX_DECLARE(389)
PRNG_RANLUX_DECLARE(120)
PRNG_RANLUX_DECLARE(240)
PRNG_RANLUX_DECLARE(408)

cudaError_t launch_fill_ranlux(const FillDesc& d, Tile t, cudaStream_t s) {
  if (d.n_rows == 0 || d.n_per == 0) return cudaSuccess;
  switch (d.p) {
    case 24: return ranlux_fill_p<24>(d, t, s);
    case 48: return ranlux_fill_p<48>(d, t, s);
    case 97: return ranlux_fill_p<97>(d, t, s);
    case 223: return ranlux_fill_p<223>(d, t, s);
    case 389: return ranlux_fill_p<389>(d, t, s);
    case 120: return ranlux_fill_p<120>(d, t, s);
    case 240: return ranlux_fill_p<240>(d, t, s);
    case 408: return ranlux_fill_p<408>(d, t, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_batch_ranlux(const BatchQueue& q, int p, Tile t, bool f32, cudaStream_t s) {
  if (q.n_items == 0) return cudaSuccess;
  switch (p) {
    case 24: return ranlux_batch_p<24>(q, t, f32, s);
    case 48: return ranlux_batch_p<48>(q, t, f32, s);
    case 97: return ranlux_batch_p<97>(q, t, f32, s);
    case 223: return ranlux_batch_p<223>(q, t, f32, s);
    case 389: return ranlux_batch_p<389>(q, t, f32, s);
    case 120: return ranlux_batch_p<120>(q, t, f32, s);
    case 240: return ranlux_batch_p<240>(q, t, f32, s);
    case 408: return ranlux_batch_p<408>(q, t, f32, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace prng
