// Entry points whose kernels are not built yet: they report
// CCM_ERR_UNSUPPORTED so callers fail loudly.
#include "ccm_internal.cuh"

using namespace ccm;

extern "C" int ccm_path_vjp(ccm_ctx*, const double*, int64_t, int32_t, const int32_t*,
                            const double*, int64_t, const double*, int32_t, const double*,
                            const double*, const double*, double*, double*, ccm_stream_t) {
  set_error("ccm_path_vjp: not built in this version");
  return CCM_ERR_UNSUPPORTED;
}

extern "C" int ccm_solve_path_batched(ccm_ctx*, int32_t, const ccm_problem*, int32_t,
                                      const double*, int32_t, double, const ccm_options*,
                                      ccm_stats*, ccm_stream_t) {
  set_error("ccm_solve_path_batched: not built in this version");
  return CCM_ERR_UNSUPPORTED;
}
