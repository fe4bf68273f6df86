// Fused forward chain: ray generation + Fourier encoding written straight
// into shared memory, then all hidden layers as tcgen05 GEMMs on chip.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "internal.cuh"

namespace dinr {

constexpr int kChainMaxLayers = 8;

struct ChainMaps {
  CUtensorMap w[kChainMaxLayers];  // BF16 weights W_L [W][K_L], box {64, W}
  CUtensorMap h[kChainMaxLayers];  // BF16 outputs h_L [samples][W], box {64, 32}
  CUtensorMap e;                   // BF16 features E [samples][ldE], box {64, 32}
};

struct ChainArgs {
  GeoDev g;
  SourceArgs src;
  long long n_rays;
  int S, F, d_in;
  int k0;                          // layer-0 K padded to a multiple of 64
  int W, H;
  long long ns;                    // samples = n_rays * S
  int m_tiles;
  int stages;
  int store_h;                     // write h_L to HBM (training) or not (queries)
  const float *bias[kChainMaxLayers];
  const float *w_out, *b_out;
  float *z_out;                    // [ns]
  float *ray_l, *ray_p;            // [n_rays]
  const float *proj;               // measured stack (training rays) or null
  int *err;
};

// Shared memory the chain needs for a width, layer-0 K and stage count.
size_t chain_smem_bytes(int W, int k0, int stages);
int chain_stages(int W, int k0);
bool chain_supports_freq(int F);
int launch_fwd_chain(const ChainMaps &maps, const ChainArgs &a, int num_sms, cudaStream_t st);

}  // namespace dinr
