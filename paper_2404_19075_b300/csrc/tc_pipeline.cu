#include "tc.cuh"

bool tc_supported(const dinr_net *) { return false; }
long long tc_bytes_per_sample(const dinr_ctx *) { return 0; }
dinr_status tc_alloc(dinr_ctx *) { return DINR_ERR_UNSUPPORTED; }
void tc_destroy(dinr_ctx *) {}
dinr_status tc_params_changed(dinr_ctx *) { return DINR_OK; }
dinr_status tc_loss_grad(dinr_ctx *, int) { return DINR_ERR_UNSUPPORTED; }
dinr_status tc_forward_rays(dinr_ctx *, const dinr::SourceArgs &, long long, int, float *) {
  return DINR_ERR_UNSUPPORTED;
}
dinr_status tc_forward_points(dinr_ctx *, const dinr::SourceArgs &, long long, float *) {
  return DINR_ERR_UNSUPPORTED;
}
