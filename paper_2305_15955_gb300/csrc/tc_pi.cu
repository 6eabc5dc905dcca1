// Placeholder until the tcgen05 kernel lands: the mixed path reports UNSUPPORTED.
#include "tc_pi.cuh"

size_t tc_pi_scratch_bytes(int, long) { return 256; }
cdwac_status tc_pi_prepare(cdwac_ctx* ctx, const void*, int, int, long, void*, cudaStream_t) {
  return set_error(ctx, CDWAC_ERR_UNSUPPORTED, "mixed precision not built");
}
cdwac_status tc_pi_imag(cdwac_ctx* ctx, void*, const double*, int, long, const double*, double*, cudaStream_t) {
  return set_error(ctx, CDWAC_ERR_UNSUPPORTED, "mixed precision not built");
}
cdwac_status tc_pi_complex(cdwac_ctx* ctx, void*, const double*, int, long, const cplx*, cplx*, cudaStream_t) {
  return set_error(ctx, CDWAC_ERR_UNSUPPORTED, "mixed precision not built");
}
