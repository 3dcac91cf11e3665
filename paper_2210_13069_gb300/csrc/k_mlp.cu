// k_mlp.cu -- the learned (n, P) selector: a 3-layer FP32 MLP with hand-written forward,
// backward and Adam kernels.
#include "lrtei_internal.h"

struct lrtei_selector {
  int hidden = 64;
};

extern "C" {
lrtei_status lrtei_selector_create(int hidden, uint64_t seed, lrtei_selector** out) {
  (void)hidden; (void)seed;
  if (out) *out = nullptr;
  lrtei::set_error("selector not built yet");
  return LRTEI_ERR_UNSUPPORTED;
}
void lrtei_selector_destroy(lrtei_selector* sel) { delete sel; }
lrtei_status lrtei_selector_train_epoch(lrtei_selector*, const float*, const float*, int, int, float, float*, void*) {
  return LRTEI_ERR_UNSUPPORTED;
}
lrtei_status lrtei_selector_forward(lrtei_selector*, const float*, float*, int, void*) { return LRTEI_ERR_UNSUPPORTED; }
lrtei_status lrtei_selector_grad(lrtei_selector*, const float*, const float*, int, float*, float*, void*) {
  return LRTEI_ERR_UNSUPPORTED;
}
int64_t lrtei_selector_nparams(const lrtei_selector*) { return 0; }
lrtei_status lrtei_selector_get_params(const lrtei_selector*, float*) { return LRTEI_ERR_UNSUPPORTED; }
lrtei_status lrtei_selector_set_params(lrtei_selector*, const float*) { return LRTEI_ERR_UNSUPPORTED; }
}
