// The context behind the opaque dinr_ctx handle, and the pipeline entry
// points the C ABI dispatches to.
#pragma once

#include "../../include/dinr.h"
#include "internal.cuh"

#include <string>
#include <vector>

// One recorded launch (or group of launches) of the context.
struct ProfRec {
  int cls;                 // index into dinr_ctx::prof_names
  cudaEvent_t a, b;
  double flops, bytes;
};

struct dinr_ctx {
  cudaStream_t st = nullptr;
  dinr::GeoDev geo{};
  double2 *d_view_cs = nullptr;
  double *d_view_tbar = nullptr, *d_view_t = nullptr;
  double t0 = 0, t1 = 1;
  int det_rows = 0, det_cols = 0, S = 1;
  float mu0 = 1.0f;

  // network: layer L = 0..H-1 hidden, L = H output; offsets into the flat vector
  int F = 0, H = 0, W = 0, act = 0, out_act = 0, prec = 0, d_in = 0, ldE = 0;
  int grff_c = 0;                  // GRFF encoding: C frequencies (0: octave encoding)
  std::vector<float> grff_B;       // host copy [C][4]
  float *d_grff_B = nullptr;       // device copy [C][4]
  long long P = 0;
  std::vector<int> fan_in, fan_out;
  std::vector<long long> offW, offb;

  float *d_params = nullptr, *d_m = nullptr, *d_v = nullptr, *d_grad = nullptr;
  float *d_loss = nullptr, *d_proj = nullptr;
  long long n_proj = 0;
  long long *d_idx = nullptr;
  int *d_flag = nullptr;

  double lr = 1e-3, b1 = 0.9, b2 = 0.999, eps = 1e-8, decay = 1.0;
  int batch_rays = 0, chunk_rays = 0;
  int recompute = 0;          // BF16 unfused path: keep checkpoints only (see dinr_train)
  uint64_t sampler_seed = 0;
  long long step = 0;  // completed Adam steps

  // The minibatch of the last dinr_forward, left for dinr_backward: its
  // rays (0: none; restaging the indices clears it) and, when the step fit
  // in one pass, its samples with the activations still in the workspace
  // (any other use of the workspace clears fwd_kept).
  int fwd_n = 0;
  bool fwd_kept = false;
  long long fwd_ns = 0;

  // FP32 workspace (per pass of chunk_rays rays)
  float *E = nullptr, *Z = nullptr, *D0 = nullptr, *D1 = nullptr;
  float *zout = nullptr, *dz = nullptr;
  float *ray_l = nullptr, *ray_p = nullptr, *pbar = nullptr, *sq = nullptr;
  float *part = nullptr;
  long long part_floats = 0;

  // Graph-replayed training steps (dinr_train_graph): one step captured
  // once per minibatch size and replayed on a private stream; the step
  // counter and a table of per-step learning rates and bias corrections
  // live in device memory while it runs.
  long long *d_step = nullptr, *d_step0 = nullptr;
  float *d_sched = nullptr;       // [sched_cap][3]
  int sched_cap = 0;
  void *gexec = nullptr;          // cudaGraphExec_t of one step
  int g_rays = 0;                 // minibatch size it was captured for
  long long g_kernels = 0;        // kernel nodes of the graph
  // the same for a step on indices already staged in d_idx (host indices
  // of dinr_train_step): no sampler kernel
  void *gexec_staged = nullptr;
  int gs_rays = 0;
  long long gs_kernels = 0;
  cudaStream_t gst = nullptr;
  cudaEvent_t gev[2] = {nullptr, nullptr};

  // BF16 (tensor-core) backend state, owned by the tensor-core pipeline.
  void *tc = nullptr;
  // query server state (serve.cu)
  void *serve = nullptr;
  void *subpix = nullptr;         // App. A sub-ray workspace (subpixel.cu)

  // per-kernel event timing (dinr_profile)
  bool prof = false;
  long long samples_done = 0;  // network samples of training passes since profiling began
  std::vector<std::string> prof_names;
  std::vector<ProfRec> prof_recs;
  std::vector<cudaEvent_t> prof_pool;
  size_t prof_used = 0;
  long long launches = 0;  // kernels launched by this context

  char err[512] = "no error";
  bool failed = false;
  std::vector<void *> allocs;
};

int dinr_fail(dinr_ctx *c, int status, const char *fmt, ...);

// Whether a geometry description is one the library accepts (the argument
// checks shared by dinr_create and the phantom projectors).
inline bool dinr_geometry_valid(const dinr_geometry *g) {
  if (!g || !g->view_angle || !g->view_time) return false;
  if (g->beam != DINR_BEAM_PARALLEL && g->beam != DINR_BEAM_CONE) return false;
  if (g->n_views < 1 || g->det_rows < 1 || g->det_cols < 1) return false;
  if (!(g->det_pitch_u > 0) || !(g->det_pitch_v > 0) || !(g->fov_r > 0)) return false;
  if (!(g->fov_z1 > g->fov_z0) || !(g->t1 > g->t0)) return false;
  if (g->samples_per_ray < 1 || g->samples_per_ray > 4096) return false;
  if (g->beam == DINR_BEAM_CONE && (!(g->sod > g->fov_r) || !(g->sdd > g->sod))) return false;
  if (g->subpixels < 0 || g->subpixels > 8) return false;
  return true;
}
void dinr_serve_release(dinr_ctx *c);

// Brackets the launches issued in its scope with two events on the context
// stream when profiling is on, and always with an NVTX range of the same
// name (free without a tool attached; ncu --nvtx and nsys pick them up).
struct ProfScope {
  dinr_ctx *c;
  int idx = -1;
  ProfScope(dinr_ctx *ctx, const char *name, double flops, double bytes);
  ~ProfScope();
};

// Pipeline (pipeline.cu)
bool bf16_supported(const dinr_net *net);
long long workspace_bytes_per_sample(const dinr_ctx *c);
// Whether activation recomputation applies to this context's path.
bool recompute_applies(const dinr_ctx *c);
dinr_status alloc_workspace(dinr_ctx *c);
void destroy_backend(dinr_ctx *c);
// What a loss-and-gradient run of the n staged rays in d_idx does:
// kLossGrad loss into d_loss and gradient into d_grad (every pass forward
// then backward); kLossOnly the forward and loss only, keeping the
// activations when the minibatch is one pass (fwd_kept, fwd_ns); kGradOnly
// the backward of the kept pass (callers recompute with kLossGrad when
// nothing was kept).
enum RunMode { kLossGrad = 0, kLossOnly = 1, kGradOnly = 2 };
dinr_status run_loss_grad(dinr_ctx *c, int n, RunMode mode = kLossGrad);
// Forward model p_bar for n_rays rays of a source, S samples each, into out.
dinr_status run_forward_rays(dinr_ctx *c, const dinr::SourceArgs &src, long long n_rays, int S,
                             float *out);
// mu0 * M at n points of a source into out.
dinr_status run_forward_points(dinr_ctx *c, const dinr::SourceArgs &src, long long n, float *out);
// Waits for the stream; reports device-side failures recorded by kernels.
dinr_status backend_poll(dinr_ctx *c);
// Refresh derived copies of the parameters (BF16 weights) after a change.
dinr_status after_param_update(dinr_ctx *c);
