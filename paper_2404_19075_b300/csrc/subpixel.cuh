// App. A forward model on the GPU: D x D sub-pixel rays per pixel with a
// variable number of samples per ray (ragged segments).
#pragma once

#include "context.cuh"

// Per pass: the sub-ray table of n_pix minibatch pixels idx (device),
// sample offsets (exclusive scan of the per-ray counts), the owner sub-ray
// of every sample and each pixel's measurement. Returns the number of
// samples of the pass on the host (one stream synchronisation).
dinr_status subpix_setup(dinr_ctx *c, const long long *idx, int n_pix, const float *proj,
                         long long *n_samples);
// Sample source of the last setup (kSrcSubRays).
dinr::SourceArgs subpix_source(dinr_ctx *c);
// Forward model (Eq. 1, App. A) and loss terms of the last setup from the
// per-sample outputs z_out: p_bar[n_pix]; when train also sq[n_pix] =
// (p_bar - p)^2 and dz[sample] = (2/B)(p_bar - p) mu0 l / |Phi| out'(z).
dinr_status subpix_segsum(dinr_ctx *c, const float *z_out, int n_pix, float inv_B, bool train,
                          float *p_bar, float *sq, float *dz);
dinr_status subpix_alloc(dinr_ctx *c);
void subpix_free(dinr_ctx *c);
