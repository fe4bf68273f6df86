// Tensor-core (tcgen05) BF16 pipeline of the training step and queries.
#pragma once

#include "context.cuh"

bool tc_supported(const dinr_net *net);
long long tc_bytes_per_sample(const dinr_ctx *c);
bool tc_recompute_applies(const dinr_ctx *c);
dinr_status tc_alloc(dinr_ctx *c);
void tc_destroy(dinr_ctx *c);
dinr_status tc_params_changed(dinr_ctx *c);
dinr_status tc_loss_grad(dinr_ctx *c, int n, RunMode mode);
dinr_status tc_forward_rays(dinr_ctx *c, const dinr::SourceArgs &src, long long n_rays, int S,
                            float *out);
dinr_status tc_forward_points(dinr_ctx *c, const dinr::SourceArgs &src, long long n, float *out);
// Waits for the stream and reports a bounded device wait that gave up.
dinr_status tc_poll(dinr_ctx *c);
