// Fused forward chain: ray generation + Fourier encoding written straight
// into shared memory, then all hidden layers as tcgen05 GEMMs on chip.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "internal.cuh"

namespace dinr {

constexpr int kChainMaxLayers = 8;
// Template value of the encoding for Gaussian random Fourier features with
// C = 128 (2C = 256 inputs); octave encodings use F itself (<= 16).
constexpr int kGrffChain = 128;
// Hidden-layer activation of a chain.
constexpr int kActRelu = 0, kActSwish = 1;

// One piece of a serving batch: samples [0, n) of a query, starting at tile
// tile0 of the batch (items start on 128-sample tile boundaries).
struct WorkItem {
  int kind;          // kSrcVirtualView (rays from records) or kSrcPoints / kSrcGrid
  int S;             // samples per ray (rays), 1 otherwise
  long long tile0;   // first tile of the item in the batch
  long long n;       // samples of the item in this batch
  long long rec0;    // first ray record of the item (rays)
  SourceArgs src;    // points / grid source, `first` = offset within the query
};

struct ChainMaps {
  // forward: BF16 weights W_L [W][K_L]; backward: transposed W_L^T [W][W]; box {64, W}
  CUtensorMap w[kChainMaxLayers];
  // forward: outputs h_L; backward: deltas delta_L; [samples][W], box {64, 32}
  CUtensorMap h[kChainMaxLayers];
  CUtensorMap e;                   // forward: features E [samples][ldE], box {64, 32}
};

struct ChainArgs {
  GeoDev g;
  SourceArgs src;
  long long n_rays;
  int S, F, d_in;
  int grff_c;                      // GRFF encoding (C = 128) or 0 (octave features)
  float grff_B[kGrffChain][4];     // frozen GRFF matrix (t, z, y, x columns)
  int k0;                          // layer-0 K padded to a multiple of 64
  int W, H;
  long long ns;                    // samples = n_rays * S
  int m_tiles;
  int stages;
  int store_h;                     // write h_L to HBM (training) or not (queries)
  // Training with every tile inside one ray and an identity output: instead
  // of storing h_{H-1} (read only by the output-layer weight gradient), the
  // forward writes, per tile and TMEM lane quadrant q, the column sums of
  // h_{H-1} (its BF16 values) over the quadrant's live rows,
  // hsum[(tile * 4 + q) * W + c]; null: h_{H-1} is stored like the others.
  float *hsum;
  const float *bias[kChainMaxLayers];
  const float *w_out, *b_out;
  float *z_out;                    // [ns]
  float *ray_l, *ray_p;            // [n_rays]
  const float *rays;               // per-ray records [n_rays][8] (ray sources), see
                                   // launch_ray_records
  const int *owner;                // App. A: ray of each sample (null: S samples per ray)
  const long long *sfirst;         // App. A: first sample of each ray
  int act;                         // kActRelu or kActSwish
  // ReLU: bits of h_L, W/32 words per sample, tile-interleaved (see
  // mask_unit in tc_chain.cu), ceil(samples / 128) * 128 * W / 32 words per layer
  uint32_t *masks[kChainMaxLayers];
  // Swish: derivative at z_L, BF16, tile-interleaved (see gact_unit in
  // tc_chain.cu), ceil(samples / 128) * 128 * W values per layer
  __nv_bfloat16 *gact[kChainMaxLayers];
  const float *proj;               // measured stack (training rays) or null
  // serving batches: per-tile work items (null for a single source)
  const WorkItem *items;
  const int *tile_item;            // [m_tiles] item of each tile
  // backward chain
  const float *dz;                 // dL/dz_out per sample
  int *err;
};

// Per-ray records for the forward chain, one thread per ray in FP64 (Sec. III
// decode and rotation, FOV chord, App. A midpoints, App. B normalisation):
// normalised time, normalised position of sample 0, normalised step between
// samples (z, y, x each) and the chord length, as FP32 [n_rays][8]; also the
// chord length and measured value of each ray.
void launch_ray_records(const GeoDev &g, const SourceArgs &src, long long n_rays, int S,
                        float *rec, float *ray_l, const float *proj, float *ray_p,
                        cudaStream_t st);

// Shared memory the chain needs for a width, layer-0 K and stage count.
size_t chain_smem_bytes(int W, int k0, int stages);
int chain_stages(int W, int k0);
bool chain_supports_freq(int F);
bool chain_supports_grff(int C);
int launch_fwd_chain(const ChainMaps &maps, const ChainArgs &a, int num_sms, cudaStream_t st);
// Backward chain (H >= 2): delta_{H-1} = dz w_out [h_{H-1} > 0], then
// delta_{L-1} = (delta_L W_L) [h_{L-1} > 0] for L = H-1..1, all on chip, with
// the ReLU bits the forward chain wrote to masks[L]; every delta_L is stored
// through maps.h[L].
int launch_bwd_chain(const ChainMaps &maps, const ChainArgs &a, int num_sms, cudaStream_t st);

}  // namespace dinr
