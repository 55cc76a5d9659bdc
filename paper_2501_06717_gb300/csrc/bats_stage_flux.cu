// bats_stage_flux.cu -- the stage kernel's instantiations with the HLL and
// the Linde flux (plain kernels, both precisions, every limiter, with and
// without an analytic B0), compiled apart from bats_stage.cu so that the two
// halves of the instantiations build in parallel.
#include "bats_stage_kernel.h"

namespace batsk {

using StageFn = void (*)(const StageArgs);
template <bool MIXED, int FLX>
static StageFn pick(int lim, bool b0) {
  if (lim == 2) return b0 ? k_stage<MIXED, 2, true, false, FLX> : k_stage<MIXED, 2, false, false, FLX>;
  if (lim == 1) return b0 ? k_stage<MIXED, 1, true, false, FLX> : k_stage<MIXED, 1, false, false, FLX>;
  return b0 ? k_stage<MIXED, 0, true, false, FLX> : k_stage<MIXED, 0, false, false, FLX>;
}
StageFn stage_fn_flux(bool mixed, int lim, bool b0, int flux) {
  if (flux == FLUX_LINDE) return mixed ? pick<true, FLUX_LINDE>(lim, b0) : pick<false, FLUX_LINDE>(lim, b0);
  return mixed ? pick<true, FLUX_HLL>(lim, b0) : pick<false, FLUX_HLL>(lim, b0);
}
// Checked build: read and clear this module's index-check flag.
cudaError_t read_index_flag_flux(int32_t* out) {
#ifdef BATS_CHECKED
  cudaError_t e = cudaMemcpyFromSymbol(out, g_index_err, sizeof(int32_t));
  const int32_t zero = 0;
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_index_err, &zero, sizeof(int32_t));
  return e;
#else
  *out = 0;
  return cudaSuccess;
#endif
}

}  // namespace batsk
