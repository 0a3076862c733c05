// batch.cu -- batched sweeps (see include/lbm.h).
#include <string>

#include "lbm.h"

struct lbm_batch {
  std::string err;
};

static std::string g_batch_err = "batched sweeps are not built yet";

extern "C" lbm_status lbm_batch_create(lbm_ctx* const* ctxs, int n, lbm_batch** out) {
  (void)ctxs;
  (void)n;
  if (out) *out = nullptr;
  return LBM_EUNSUPPORTED;
}
extern "C" lbm_status lbm_batch_step(lbm_batch* b, int nsteps) {
  (void)b;
  (void)nsteps;
  return LBM_EUNSUPPORTED;
}
extern "C" lbm_status lbm_batch_tune(lbm_batch* b, int best[2]) {
  (void)b;
  (void)best;
  return LBM_EUNSUPPORTED;
}
extern "C" void lbm_batch_destroy(lbm_batch* b) { delete b; }
extern "C" const char* lbm_batch_last_error(const lbm_batch* b) {
  return b ? b->err.c_str() : g_batch_err.c_str();
}
