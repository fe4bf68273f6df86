// C ABI of libdinr (include/dinr.h): context management, argument checks,
// and dispatch to the step / query pipelines.
#include "context.cuh"

#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

using namespace dinr;

static char g_create_error[512] = "no error";

int dinr_fail(dinr_ctx *c, int status, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) {
    snprintf(c->err, sizeof(c->err), "%s", buf);
    if (status == DINR_ERR_CUDA) c->failed = true;
  } else {
    snprintf(g_create_error, sizeof(g_create_error), "%s", buf);
  }
  return status;
}

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return (dinr_status)dinr_fail(c, DINR_ERR_CUDA, "%s: %s (%s:%d)", #call,        \
                                    cudaGetErrorString(e_), __FILE__, __LINE__);      \
  } while (0)
#define CKL()            \
  do {                   \
    ++c->launches;       \
    CK(cudaGetLastError()); \
  } while (0)
#define LIVE(c)                                                                       \
  do {                                                                                \
    if (!(c)) return DINR_ERR_ARG;                                                    \
    if ((c)->failed) return DINR_ERR_CUDA;                                            \
  } while (0)

// ------------------------------------------------------------ helpers

int64_t dinr_param_count_din(int d_in, int hidden_layers, int width) {
  if (d_in < 1 || hidden_layers < 1 || width < 1) return -1;
  int64_t W = width;
  return W * d_in + W + (int64_t)(hidden_layers - 1) * (W * W + W) + W + 1;
}

int64_t dinr_param_count(int n_freq, int hidden_layers, int width) {
  if (n_freq < 0) return -1;
  return dinr_param_count_din(4 + 8 * n_freq, hidden_layers, width);
}

// He initialisation: SplitMix64 stream of `seed`, Box-Muller pairs (u1 from
// (0,1]); weight entries in layout order take consecutive normals scaled by
// sqrt(2/fan_in); biases are 0.
static void he_init_host(const dinr_ctx *c, uint64_t seed, std::vector<float> &out) {
  out.assign(c->P, 0.0f);
  uint64_t k = 0;
  auto uni = [&]() {
    ++k;
    return (double)(mix64(seed + k * kGamma) >> 11) * (1.0 / 9007199254740992.0);
  };
  double spare = 0.0;
  bool have = false;
  auto normal = [&]() {
    if (have) {
      have = false;
      return spare;
    }
    double u1 = 1.0 - uni(), u2 = uni();
    double r = std::sqrt(-2.0 * std::log(u1));
    spare = r * std::sin(2.0 * M_PI * u2);
    have = true;
    return r * std::cos(2.0 * M_PI * u2);
  };
  for (int L = 0; L <= c->H; ++L) {
    int64_t fo = c->fan_out[L], fi = c->fan_in[L];
    double sd = std::sqrt(2.0 / (double)fi);
    for (int64_t q = 0; q < fo * fi; ++q) out[c->offW[L] + q] = (float)(normal() * sd);
  }
}

static void *dev_alloc(dinr_ctx *c, size_t bytes, bool *ok) {
  void *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *ok = false;
    return nullptr;
  }
  c->allocs.push_back(p);
  return p;
}

// Device geometry tables from the host description (FP64, per view).
static dinr_status setup_geometry(dinr_ctx *c, const dinr_geometry *g, GeoDev *geo,
                                  double2 **cs_out, double **tbar_out, double **t_out,
                                  cudaStream_t st) {
  int M = g->n_views;
  std::vector<double2> cs(M);
  std::vector<double> tb(M), tt(M);
  for (int m = 0; m < M; ++m) {
    cs[m] = make_double2(std::cos(g->view_angle[m]), std::sin(g->view_angle[m]));
    tt[m] = g->view_time[m];
    tb[m] = 2.0 * (g->view_time[m] - g->t0) / (g->t1 - g->t0) - 1.0;
  }
  bool ok = true;
  *cs_out = (double2 *)dev_alloc(c, sizeof(double2) * M, &ok);
  *tbar_out = (double *)dev_alloc(c, sizeof(double) * M, &ok);
  *t_out = (double *)dev_alloc(c, sizeof(double) * M, &ok);
  if (!ok) return (dinr_status)dinr_fail(c, DINR_ERR_OOM, "geometry tables: out of memory");
  CK(cudaMemcpyAsync(*cs_out, cs.data(), sizeof(double2) * M, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(*tbar_out, tb.data(), sizeof(double) * M, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(*t_out, tt.data(), sizeof(double) * M, cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  GeoDev &d = *geo;
  d.beam = g->beam;
  d.n_views = g->n_views;
  d.det_rows = g->det_rows;
  d.det_cols = g->det_cols;
  d.n_pixels = (long long)g->det_rows * g->det_cols;
  d.n_proj = d.n_pixels * g->n_views;
  d.pu = g->det_pitch_u;
  d.pv = g->det_pitch_v;
  d.ou = g->det_off_u;
  d.ov = g->det_off_v;
  d.sod = g->sod;
  d.sdd = g->sdd;
  d.R = g->fov_r;
  d.z0 = g->fov_z0;
  d.z1 = g->fov_z1;
  d.inv_R = 1.0 / g->fov_r;
  d.zs = 2.0 / (g->fov_z1 - g->fov_z0);
  d.zb = -(g->fov_z0 + g->fov_z1) / (g->fov_z1 - g->fov_z0);
  d.S = g->samples_per_ray;
  d.D = g->subpixels;
  d.spacing = 0.0;
  if (d.D > 0) {
    double pitch = g->det_pitch_u < g->det_pitch_v ? g->det_pitch_u : g->det_pitch_v;
    if (g->beam == DINR_BEAM_CONE) pitch *= g->sod / g->sdd;
    d.spacing = pitch / d.D;
  }
  d.mu0 = (float)g->mu0;
  d.view_cs = *cs_out;
  d.view_tbar = *tbar_out;
  return DINR_OK;
}

// ------------------------------------------------------------- create

static dinr_status create_fail(dinr_ctx *c, dinr_status s) {
  if (c) {
    snprintf(g_create_error, sizeof(g_create_error), "%s", c->err);
    dinr_destroy(c);
  }
  return s;
}

dinr_status dinr_create(const dinr_geometry *geom, const dinr_net *net, const dinr_train *train,
                        const float *proj, int proj_on_device, void *cuda_stream,
                        dinr_ctx **out) {
  if (!out) return (dinr_status)dinr_fail(nullptr, DINR_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!dinr_geometry_valid(geom))
    return (dinr_status)dinr_fail(nullptr, DINR_ERR_ARG, "invalid geometry");
  if (!net || net->n_freq < 0 || net->n_freq > kMaxFreq || net->hidden_layers < 1 ||
      net->hidden_layers > 32 || net->width < 1 || net->width > 1024 ||
      (net->act != DINR_ACT_RELU && net->act != DINR_ACT_SWISH) ||
      (net->out_act != DINR_OUT_IDENTITY && net->out_act != DINR_OUT_SOFTPLUS))
    return (dinr_status)dinr_fail(nullptr, DINR_ERR_ARG, "invalid network shape");
  if (net->encoding != DINR_ENC_OCTAVE &&
      (net->encoding != DINR_ENC_GRFF || net->grff_c < 2 || net->grff_c > kMaxGrff ||
       net->grff_c % 2 != 0 || !net->grff_B))
    return (dinr_status)dinr_fail(nullptr, DINR_ERR_ARG, "invalid encoding");
  if (net->prec != DINR_PREC_FP32 && net->prec != DINR_PREC_BF16 && net->prec != DINR_PREC_FP8)
    return (dinr_status)dinr_fail(nullptr, DINR_ERR_ARG, "invalid precision");
  if (!train || train->batch_rays < 1 || train->chunk_rays < 0)
    return (dinr_status)dinr_fail(nullptr, DINR_ERR_ARG, "invalid training options");
  if (!proj) return (dinr_status)dinr_fail(nullptr, DINR_ERR_ARG, "proj is NULL");
  if (net->prec != DINR_PREC_FP32 && !bf16_supported(net))
    return (dinr_status)dinr_fail(nullptr, DINR_ERR_UNSUPPORTED,
                                  "the tensor-core paths do not support this network shape");

  cudaGetLastError();  // a stale error of an earlier call is not this context's
  dinr_ctx *c = new (std::nothrow) dinr_ctx();
  if (!c) return (dinr_status)dinr_fail(nullptr, DINR_ERR_OOM, "host allocation failed");
  c->st = (cudaStream_t)cuda_stream;
  cudaStream_t st = c->st;
  c->F = net->n_freq;
  c->H = net->hidden_layers;
  c->W = net->width;
  c->act = net->act;
  c->out_act = net->out_act;
  c->prec = net->prec;
  c->d_in = 4 + 8 * c->F;
  if (net->encoding == DINR_ENC_GRFF) {
    c->grff_c = net->grff_c;
    c->grff_B.assign(net->grff_B, net->grff_B + 4 * net->grff_c);
    c->d_in = 2 * c->grff_c;
  }
  c->ldE = (c->d_in + 15) / 16 * 16;
  c->S = geom->samples_per_ray;
  c->mu0 = (float)geom->mu0;
  c->det_rows = geom->det_rows;
  c->det_cols = geom->det_cols;
  c->t0 = geom->t0;
  c->t1 = geom->t1;
  long long off = 0;
  for (int L = 0; L <= c->H; ++L) {
    int fi = L == 0 ? c->d_in : c->W, fo = L == c->H ? 1 : c->W;
    c->fan_in.push_back(fi);
    c->fan_out.push_back(fo);
    c->offW.push_back(off);
    off += (long long)fi * fo;
    c->offb.push_back(off);
    off += fo;
  }
  c->P = off;
  c->lr = train->lr > 0 ? train->lr : 1e-3;
  c->b1 = train->beta1 > 0 ? train->beta1 : 0.9;
  c->b2 = train->beta2 > 0 ? train->beta2 : 0.999;
  c->eps = train->eps > 0 ? train->eps : 1e-8;
  c->decay = train->lr_decay_per_epoch > 0 ? train->lr_decay_per_epoch : 1.0;
  c->batch_rays = train->batch_rays;
  c->sampler_seed = train->sampler_seed;

  dinr_status s = setup_geometry(c, geom, &c->geo, &c->d_view_cs, &c->d_view_tbar,
                                 &c->d_view_t, st);
  if (s != DINR_OK) return create_fail(c, s);
  if (c->geo.D > 0) {
    // App. A: workspaces hold the most samples a pixel can have, D^2 rays of
    // ceil(longest chord / spacing) samples (longest chord: the cylinder's
    // diagonal)
    const double R = geom->fov_r, hz = geom->fov_z1 - geom->fov_z0;
    const double lmax = std::sqrt(4.0 * R * R + hz * hz);
    c->S = c->geo.D * c->geo.D * ((int)std::ceil(lmax / c->geo.spacing) + 1);
  }
  c->n_proj = c->geo.n_proj;

  bool ok = true;
  c->d_params = (float *)dev_alloc(c, sizeof(float) * c->P, &ok);
  c->d_m = (float *)dev_alloc(c, sizeof(float) * c->P, &ok);
  c->d_v = (float *)dev_alloc(c, sizeof(float) * c->P, &ok);
  c->d_grad = (float *)dev_alloc(c, sizeof(float) * c->P, &ok);
  c->d_loss = (float *)dev_alloc(c, sizeof(float) * 4, &ok);
  c->d_proj = (float *)dev_alloc(c, sizeof(float) * c->n_proj, &ok);
  c->d_idx = (long long *)dev_alloc(c, sizeof(long long) * c->batch_rays, &ok);
  c->d_flag = (int *)dev_alloc(c, sizeof(int) * 4, &ok);
  if (c->grff_c > 0) c->d_grff_B = (float *)dev_alloc(c, sizeof(float) * 4 * c->grff_c, &ok);
  if (!ok) {
    dinr_fail(c, DINR_ERR_OOM, "device allocation of parameters/projections failed");
    return create_fail(c, DINR_ERR_OOM);
  }
  std::vector<float> init;
  const float *src = net->init_params;
  if (!src) {
    he_init_host(c, net->seed, init);
    src = init.data();
  }
  CK(cudaMemcpyAsync(c->d_params, src, sizeof(float) * c->P, cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(c->d_m, 0, sizeof(float) * c->P, st));
  CK(cudaMemsetAsync(c->d_v, 0, sizeof(float) * c->P, st));
  CK(cudaMemsetAsync(c->d_grad, 0, sizeof(float) * c->P, st));
  CK(cudaMemsetAsync(c->d_loss, 0, sizeof(float) * 4, st));
  CK(cudaMemsetAsync(c->d_flag, 0, sizeof(int) * 4, st));
  if (c->grff_c > 0)
    CK(cudaMemcpyAsync(c->d_grff_B, c->grff_B.data(), sizeof(float) * 4 * c->grff_c,
                       cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(c->d_proj, proj, sizeof(float) * c->n_proj,
                     proj_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));

  // Rays per pass: bounded so that the activations of a pass fit in a
  // workspace budget of 60 % of free memory, at most 96 GiB.
  size_t free_b = 0, total_b = 0;
  CK(cudaMemGetInfo(&free_b, &total_b));
  long long budget = (long long)(free_b * 0.6);
  if (budget > (96LL << 30)) budget = 96LL << 30;
  c->recompute = 0;
  long long max_rays = budget / (workspace_bytes_per_sample(c) * c->S + 64);
  if (recompute_applies(c) &&
      (train->recompute > 0 || (train->recompute < 0 && max_rays < c->batch_rays))) {
    c->recompute = 1;
    max_rays = budget / (workspace_bytes_per_sample(c) * c->S + 64);
  }
  long long chunk = train->chunk_rays > 0 ? train->chunk_rays : c->batch_rays;
  if (chunk > c->batch_rays) chunk = c->batch_rays;
  if (chunk > max_rays) chunk = max_rays;
  if (chunk < 1) {
    dinr_fail(c, DINR_ERR_OOM, "not enough device memory for one ray");
    return create_fail(c, DINR_ERR_OOM);
  }
  c->chunk_rays = (int)chunk;
  s = alloc_workspace(c);
  if (s != DINR_OK) return create_fail(c, s);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    dinr_fail(c, DINR_ERR_CUDA, "create: %s", cudaGetErrorString(e));
    return create_fail(c, DINR_ERR_CUDA);
  }
  *out = c;
  return DINR_OK;
}

void dinr_destroy(dinr_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->st);
  dinr_serve_release(c);
  if (c->gst) cudaStreamSynchronize(c->gst);  // replays in flight finish first
  if (c->gexec) cudaGraphExecDestroy((cudaGraphExec_t)c->gexec);
  if (c->gexec_staged) cudaGraphExecDestroy((cudaGraphExec_t)c->gexec_staged);
  for (cudaEvent_t e : c->gev)
    if (e) cudaEventDestroy(e);
  if (c->gst) cudaStreamDestroy(c->gst);
  destroy_backend(c);
  for (cudaEvent_t e : c->prof_pool) cudaEventDestroy(e);
  for (void *p : c->allocs) cudaFree(p);
  delete c;
}

const char *dinr_last_error(const dinr_ctx *c) { return c ? c->err : g_create_error; }

dinr_status dinr_synchronize(dinr_ctx *c) {
  LIVE(c);
  return backend_poll(c);
}

dinr_status dinr_set_projections(dinr_ctx *c, const float *proj, int on_device) {
  LIVE(c);
  if (!proj) return (dinr_status)dinr_fail(c, DINR_ERR_ARG, "proj is NULL");
  CK(cudaMemcpyAsync(c->d_proj, proj, sizeof(float) * c->n_proj,
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->st));
  return DINR_OK;
}

// Stage the minibatch indices into the context (sampler, host or device).
static dinr_status stage_indices(dinr_ctx *c, const int64_t *idx, int n, int on_device) {
  if (n < 1 || n > c->batch_rays)
    return (dinr_status)dinr_fail(c, DINR_ERR_ARG, "n = %d outside [1, %d]", n, c->batch_rays);
  c->fwd_n = 0;  // the minibatch a dinr_forward left is replaced
  c->fwd_kept = false;
  if (!idx) {
    launch_sample_indices(c->n_proj, n, c->step, c->sampler_seed, c->d_idx, c->st);
    CKL();
  } else if (!on_device) {
    for (int i = 0; i < n; ++i)
      if (idx[i] < 0 || idx[i] >= c->n_proj)
        return (dinr_status)dinr_fail(c, DINR_ERR_ARG, "ray index %lld outside [0, %lld)",
                                      (long long)idx[i], c->n_proj);
    CK(cudaMemcpyAsync(c->d_idx, idx, sizeof(long long) * n, cudaMemcpyHostToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));
  } else {
    CK(cudaMemcpyAsync(c->d_idx, idx, sizeof(long long) * n, cudaMemcpyDeviceToDevice, c->st));
    // Out-of-range device indices are replaced by 0 and flagged, so that no
    // kernel reads outside the view tables or the projection stack.
    launch_check_indices(c->d_idx, n, c->n_proj, c->d_flag, c->st);
    CKL();
  }
  return DINR_OK;
}

static dinr_status check_flag(dinr_ctx *c) {
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (bad) {
    CK(cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->st));
    return (dinr_status)dinr_fail(c, DINR_ERR_ARG, "a device ray index was outside [0, M*N)");
  }
  return DINR_OK;
}

dinr_status dinr_loss_grad(dinr_ctx *c, const int64_t *idx, int n, int on_device,
                           float *loss_dev, float *grad_dev) {
  LIVE(c);
  dinr_status s = stage_indices(c, idx, n, on_device);
  if (s != DINR_OK) return s;
  s = run_loss_grad(c, n);
  if (s != DINR_OK) return s;
  if (loss_dev)
    CK(cudaMemcpyAsync(loss_dev, c->d_loss, sizeof(float), cudaMemcpyDeviceToDevice, c->st));
  if (grad_dev)
    CK(cudaMemcpyAsync(grad_dev, c->d_grad, sizeof(float) * c->P, cudaMemcpyDeviceToDevice,
                       c->st));
  return DINR_OK;
}

dinr_status dinr_forward(dinr_ctx *c, const int64_t *idx, int n, int on_device,
                         float *loss_dev) {
  LIVE(c);
  dinr_status s = stage_indices(c, idx, n, on_device);
  if (s != DINR_OK) return s;
  s = run_loss_grad(c, n, kLossOnly);
  if (s != DINR_OK) return s;
  c->fwd_n = n;
  if (loss_dev)
    CK(cudaMemcpyAsync(loss_dev, c->d_loss, sizeof(float), cudaMemcpyDeviceToDevice, c->st));
  return DINR_OK;
}

dinr_status dinr_backward(dinr_ctx *c, const float *dloss_dev, float *grad_dev) {
  LIVE(c);
  if (c->fwd_n < 1)
    return (dinr_status)dinr_fail(c, DINR_ERR_ARG,
                                  "dinr_backward: no dinr_forward minibatch to differentiate");
  // the kept activations of a one-pass forward, else the whole step again
  dinr_status s = run_loss_grad(c, c->fwd_n, c->fwd_kept ? kGradOnly : kLossGrad);
  if (s != DINR_OK) return s;
  if (dloss_dev) {
    launch_scale_by(c->d_grad, c->P, dloss_dev, c->d_grad, c->st);
    CKL();
  }
  if (grad_dev)
    CK(cudaMemcpyAsync(grad_dev, c->d_grad, sizeof(float) * c->P, cudaMemcpyDeviceToDevice,
                       c->st));
  return DINR_OK;
}

static dinr_status train_step_staged(dinr_ctx *c, const int64_t *idx, int n, float *loss_out);

dinr_status dinr_train_step(dinr_ctx *c, const int64_t *idx, int n, int on_device,
                            float *loss_out) {
  LIVE(c);
  // host indices with the loss read back: one graph launch per step (not
  // for App. A passes, which read sample counts back, or when profiling,
  // which times every launch)
  if (idx && !on_device && loss_out && c->geo.D == 0 && !c->prof)
    return train_step_staged(c, idx, n, loss_out);
  dinr_status s = stage_indices(c, idx, n, on_device);
  if (s != DINR_OK) return s;
  s = run_loss_grad(c, n);
  if (s != DINR_OK) return s;
  // Adam step t = step + 1 with bias corrections and the epoch's learning rate.
  long long t = c->step + 1;
  long long spe = (c->n_proj + n - 1) / n;
  double lr = c->lr * std::pow(c->decay, (double)(c->step / spe));
  double bc1 = 1.0 / (1.0 - std::pow(c->b1, (double)t));
  double bc2 = 1.0 / (1.0 - std::pow(c->b2, (double)t));
  {
    ProfScope ps(c, "adam", 0.0, 28.0 * c->P);
    launch_adam(c->d_params, c->d_m, c->d_v, c->d_grad, c->P, (float)lr, (float)c->b1,
                (float)c->b2, (float)c->eps, (float)bc1, (float)bc2, c->st);
    CKL();
  }
  s = after_param_update(c);
  if (s != DINR_OK) return s;
  c->step = t;
  if (idx && on_device && loss_out) {
    s = check_flag(c);
    if (s != DINR_OK) return s;
  }
  if (loss_out) {
    CK(cudaMemcpyAsync(loss_out, c->d_loss, sizeof(float), cudaMemcpyDeviceToHost, c->st));
    s = backend_poll(c);
    if (s != DINR_OK) return s;
    if (!std::isfinite(*loss_out))
      return (dinr_status)dinr_fail(c, DINR_ERR_NONFINITE, "loss is not finite");
  }
  return DINR_OK;
}

// The learning rate and Adam bias corrections of step `step` (0-based; Adam
// step t = step + 1), as dinr_train_step computes them.
static void step_scalars(const dinr_ctx *c, long long step, int n, float *out) {
  const long long spe = (c->n_proj + n - 1) / n;
  const long long t = step + 1;
  out[0] = (float)(c->lr * std::pow(c->decay, (double)(step / spe)));
  out[1] = (float)(1.0 / (1.0 - std::pow(c->b1, (double)t)));
  out[2] = (float)(1.0 / (1.0 - std::pow(c->b2, (double)t)));
}

// Captures one training step of n sampled rays on the private stream: the
// sampler reading the device step counter, loss and gradient, Adam from
// the table, the parameter copies, the counter's increment.
// Capture one training step of n rays into a graph: with `sampled` its
// minibatch comes from the device sampler (dinr_train_graph), otherwise
// from the indices already staged in d_idx (host indices of
// dinr_train_step).
static dinr_status capture_step(dinr_ctx *c, int n, bool sampled) {
  if (!c->gst) {
    CK(cudaStreamCreateWithFlags(&c->gst, cudaStreamNonBlocking));
    for (cudaEvent_t &e : c->gev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  void *&slot = sampled ? c->gexec : c->gexec_staged;
  if (slot) {
    cudaGraphExecDestroy((cudaGraphExec_t)slot);
    slot = nullptr;
  }
  cudaStream_t user = c->st;
  const long long launches = c->launches;  // captured launches run only when replayed
  c->st = c->gst;
  cudaError_t e = cudaStreamBeginCapture(c->gst, cudaStreamCaptureModeRelaxed);
  dinr_status s = DINR_OK;
  if (e == cudaSuccess) {
    if (sampled) {
      launch_sample_indices_dev(c->n_proj, n, c->d_step, c->sampler_seed, c->d_idx, c->st);
      ++c->launches;
    }
    s = run_loss_grad(c, n);
    if (s == DINR_OK) {
      launch_adam_tab(c->d_params, c->d_m, c->d_v, c->d_grad, c->P, (float)c->b1, (float)c->b2,
                      (float)c->eps, c->d_sched, c->d_step, c->d_step0, c->st);
      ++c->launches;
      s = after_param_update(c);
    }
    if (s == DINR_OK) {
      launch_step_inc(c->d_step, c->st);
      ++c->launches;
    }
  }
  cudaGraph_t g = nullptr;
  cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(c->gst, &g) : e;
  c->st = user;
  c->launches = launches;
  if (s != DINR_OK || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    if (s != DINR_OK) return s;
    return (dinr_status)dinr_fail(c, DINR_ERR_CUDA, "step capture: %s", cudaGetErrorString(e2));
  }
  size_t nn = 0;
  std::vector<cudaGraphNode_t> nodes;
  e = cudaGraphGetNodes(g, nullptr, &nn);
  if (e == cudaSuccess) {
    nodes.resize(nn);
    e = cudaGraphGetNodes(g, nodes.data(), &nn);
  }
  long long kernels = 0;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType ty;
    if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++kernels;
  }
  cudaGraphExec_t ex = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess)
    return (dinr_status)dinr_fail(c, DINR_ERR_CUDA, "step graph: %s", cudaGetErrorString(e));
  slot = ex;
  (sampled ? c->g_rays : c->gs_rays) = n;
  (sampled ? c->g_kernels : c->gs_kernels) = kernels;
  return DINR_OK;
}

// The device step counter and the Adam scalar table of graph-replayed steps
// (room for at least `steps` steps).
static dinr_status graph_state(dinr_ctx *c, int steps) {
  bool ok = true;
  if (!c->d_step) {
    c->d_step = (long long *)dev_alloc(c, 2 * sizeof(long long), &ok);
    if (ok) c->d_step0 = c->d_step + 1;
  }
  if (ok && steps > c->sched_cap) {
    const int cap = steps > 1024 ? steps : 1024;
    c->d_sched = (float *)dev_alloc(c, sizeof(float) * 3 * (size_t)cap, &ok);
    if (ok) c->sched_cap = cap;
  }
  if (!ok) return (dinr_status)dinr_fail(c, DINR_ERR_OOM, "step graph state: out of memory");
  return DINR_OK;
}

// dinr_train_step with host indices and the loss read back: the indices are
// copied in, then the step is replayed from a graph captured once per
// minibatch size (the same kernels, in the same order, as the ordinary
// step: bitwise the same result, without a launch per kernel per step).
static dinr_status train_step_staged(dinr_ctx *c, const int64_t *idx, int n, float *loss_out) {
  if (n < 1 || n > c->batch_rays)
    return (dinr_status)dinr_fail(c, DINR_ERR_ARG, "n = %d outside [1, %d]", n, c->batch_rays);
  for (int i = 0; i < n; ++i)
    if (idx[i] < 0 || idx[i] >= c->n_proj)
      return (dinr_status)dinr_fail(c, DINR_ERR_ARG, "ray index %lld outside [0, %lld)",
                                    (long long)idx[i], c->n_proj);
  c->fwd_n = 0;
  c->fwd_kept = false;
  dinr_status s = graph_state(c, 1);
  if (s != DINR_OK) return s;
  // the caller's indices may sit in pinned memory, whose copy runs later:
  // this call returns only after the step (and so the copy) has completed
  CK(cudaMemcpyAsync(c->d_idx, idx, sizeof(long long) * n, cudaMemcpyHostToDevice, c->st));
  float tab[3];
  step_scalars(c, c->step, n, tab);
  const long long s0[2] = {c->step, c->step};
  // pageable host sources: each copy has taken its bytes when it returns
  CK(cudaMemcpyAsync(c->d_sched, tab, sizeof(tab), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->d_step, s0, sizeof(s0), cudaMemcpyHostToDevice, c->st));
  if (!c->gexec_staged || c->gs_rays != n) {
    s = capture_step(c, n, false);
    if (s != DINR_OK) return s;
  }
  CK(cudaEventRecord(c->gev[0], c->st));
  CK(cudaStreamWaitEvent(c->gst, c->gev[0], 0));
  CK(cudaGraphLaunch((cudaGraphExec_t)c->gexec_staged, c->gst));
  CK(cudaEventRecord(c->gev[1], c->gst));
  CK(cudaStreamWaitEvent(c->st, c->gev[1], 0));
  c->step += 1;
  c->launches += c->gs_kernels;
  CK(cudaMemcpyAsync(loss_out, c->d_loss, sizeof(float), cudaMemcpyDeviceToHost, c->st));
  s = backend_poll(c);
  if (s != DINR_OK) return s;
  if (!std::isfinite(*loss_out))
    return (dinr_status)dinr_fail(c, DINR_ERR_NONFINITE, "loss is not finite");
  return DINR_OK;
}

dinr_status dinr_train_graph(dinr_ctx *c, int n, int steps, float *loss_out) {
  LIVE(c);
  if (n < 1 || n > c->batch_rays || steps < 1)
    return (dinr_status)dinr_fail(c, DINR_ERR_ARG, "n = %d outside [1, %d] or steps = %d < 1", n,
                                  c->batch_rays, steps);
  if (c->geo.D > 0 || c->prof) {
    // App. A steps read each pass's sample count back to the host, and
    // profiling times every launch: both run as ordinary steps
    for (int k = 0; k < steps; ++k) {
      dinr_status s = dinr_train_step(c, nullptr, n, 0, k + 1 == steps ? loss_out : nullptr);
      if (s != DINR_OK) return s;
    }
    return DINR_OK;
  }
  c->fwd_n = 0;  // the graph restages the minibatch indices
  c->fwd_kept = false;
  dinr_status gs = graph_state(c, steps);
  if (gs != DINR_OK) return gs;
  std::vector<float> tab(3 * (size_t)steps);
  for (int k = 0; k < steps; ++k) step_scalars(c, c->step + k, n, &tab[3 * (size_t)k]);
  const long long s0[2] = {c->step, c->step};
  // pageable host sources: each copy has taken its bytes when the call returns
  CK(cudaMemcpyAsync(c->d_sched, tab.data(), sizeof(float) * tab.size(), cudaMemcpyHostToDevice,
                     c->st));
  CK(cudaMemcpyAsync(c->d_step, s0, sizeof(s0), cudaMemcpyHostToDevice, c->st));
  if (!c->gexec || c->g_rays != n) {
    dinr_status s = capture_step(c, n, true);
    if (s != DINR_OK) return s;
  }
  CK(cudaEventRecord(c->gev[0], c->st));
  CK(cudaStreamWaitEvent(c->gst, c->gev[0], 0));
  for (int k = 0; k < steps; ++k) CK(cudaGraphLaunch((cudaGraphExec_t)c->gexec, c->gst));
  CK(cudaEventRecord(c->gev[1], c->gst));
  CK(cudaStreamWaitEvent(c->st, c->gev[1], 0));
  c->step += steps;
  c->launches += c->g_kernels * steps;
  if (loss_out) {
    CK(cudaMemcpyAsync(loss_out, c->d_loss, sizeof(float), cudaMemcpyDeviceToHost, c->st));
    dinr_status s = backend_poll(c);
    if (s != DINR_OK) return s;
    if (!std::isfinite(*loss_out))
      return (dinr_status)dinr_fail(c, DINR_ERR_NONFINITE, "loss is not finite");
  }
  return DINR_OK;
}

dinr_status dinr_predict(dinr_ctx *c, const int64_t *idx, int n, int on_device, float *pbar) {
  LIVE(c);
  if (!pbar) return (dinr_status)dinr_fail(c, DINR_ERR_ARG, "pbar is NULL");
  dinr_status s = stage_indices(c, idx, n, on_device);
  if (s != DINR_OK) return s;
  SourceArgs src{};
  src.kind = kSrcTrainRays;
  src.idx = c->d_idx;
  return run_forward_rays(c, src, n, c->S, pbar);
}

dinr_status dinr_project(dinr_ctx *c, double theta, double t, int rows, int cols, int S,
                         float *out) {
  LIVE(c);
  if (!out || rows < 1 || cols < 1 || S < 1 || S > 4096 ||
      (long long)rows * cols * S > (1LL << 31))
    return (dinr_status)dinr_fail(c, DINR_ERR_ARG, "invalid projection request");
  SourceArgs src{};
  src.kind = kSrcVirtualView;
  src.vc = std::cos(theta);
  src.vs = std::sin(theta);
  src.vtbar = 2.0 * (t - c->t0) / (c->t1 - c->t0) - 1.0;
  src.vpu = c->geo.pu * c->det_cols / cols;
  src.vpv = c->geo.pv * c->det_rows / rows;
  src.vrows = rows;
  src.vcols = cols;
  return run_forward_rays(c, src, (long long)rows * cols, S, out);
}

dinr_status dinr_query(dinr_ctx *c, const float *coords, int64_t n, float *out) {
  LIVE(c);
  if (!coords || !out || n < 0) return (dinr_status)dinr_fail(c, DINR_ERR_ARG, "invalid query");
  if (n == 0) return DINR_OK;
  SourceArgs src{};
  src.kind = kSrcPoints;
  src.points = coords;
  src.t_scale = 2.0 / (c->t1 - c->t0);
  src.t_bias = -2.0 * c->t0 / (c->t1 - c->t0) - 1.0;
  return run_forward_points(c, src, n, out);
}

dinr_status dinr_query_grid(dinr_ctx *c, double t, const double *lo, const double *hi,
                            const int *dims, float *out) {
  LIVE(c);
  if (!lo || !hi || !dims || !out || dims[0] < 1 || dims[1] < 1 || dims[2] < 1)
    return (dinr_status)dinr_fail(c, DINR_ERR_ARG, "invalid grid query");
  SourceArgs src{};
  src.kind = kSrcGrid;
  for (int d = 0; d < 3; ++d) {
    src.glo[d] = lo[d];
    src.gstep[d] = (hi[d] - lo[d]) / dims[d];
    src.gdims[d] = dims[d];
  }
  src.gtbar = 2.0 * (t - c->t0) / (c->t1 - c->t0) - 1.0;
  long long n = (long long)dims[0] * dims[1] * dims[2];
  return run_forward_points(c, src, n, out);
}

dinr_status dinr_set_params(dinr_ctx *c, const float *p, int on_device) {
  LIVE(c);
  if (!p) return (dinr_status)dinr_fail(c, DINR_ERR_ARG, "params is NULL");
  CK(cudaMemcpyAsync(c->d_params, p, sizeof(float) * c->P,
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->st));
  return after_param_update(c);
}

dinr_status dinr_get_params(dinr_ctx *c, float *p, int on_device) {
  LIVE(c);
  if (!p) return (dinr_status)dinr_fail(c, DINR_ERR_ARG, "params is NULL");
  CK(cudaMemcpyAsync(p, c->d_params, sizeof(float) * c->P,
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st));
  if (!on_device) CK(cudaStreamSynchronize(c->st));
  return DINR_OK;
}

dinr_status dinr_get_grads(dinr_ctx *c, float *host) {
  LIVE(c);
  if (!host) return (dinr_status)dinr_fail(c, DINR_ERR_ARG, "host is NULL");
  CK(cudaMemcpyAsync(host, c->d_grad, sizeof(float) * c->P, cudaMemcpyDeviceToHost, c->st));
  return backend_poll(c);
}

dinr_status dinr_get_loss(dinr_ctx *c, float *host) {
  LIVE(c);
  if (!host) return (dinr_status)dinr_fail(c, DINR_ERR_ARG, "host is NULL");
  CK(cudaMemcpyAsync(host, c->d_loss, sizeof(float), cudaMemcpyDeviceToHost, c->st));
  return backend_poll(c);
}

// ------------------------------------------------------------ state blob
struct StateHeader {
  char magic[8];
  int32_t version, F, H, W;
  int64_t P, step;
  uint64_t sampler_seed;
};

dinr_status dinr_get_state(dinr_ctx *c, void *buf, size_t *bytes) {
  LIVE(c);
  if (!bytes) return (dinr_status)dinr_fail(c, DINR_ERR_ARG, "bytes is NULL");
  size_t need = sizeof(StateHeader) + 3 * sizeof(float) * c->P;
  if (!buf) {
    *bytes = need;
    return DINR_OK;
  }
  if (*bytes < need) return (dinr_status)dinr_fail(c, DINR_ERR_ARG, "buffer too small");
  StateHeader h{};
  memcpy(h.magic, "DINRST1", 8);
  h.version = 1;
  h.F = c->F;
  h.H = c->H;
  h.W = c->W;
  h.P = c->P;
  h.step = c->step;
  h.sampler_seed = c->sampler_seed;
  char *b = (char *)buf;
  memcpy(b, &h, sizeof(h));
  float *f = (float *)(b + sizeof(h));
  CK(cudaMemcpyAsync(f, c->d_params, sizeof(float) * c->P, cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(f + c->P, c->d_m, sizeof(float) * c->P, cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(f + 2 * c->P, c->d_v, sizeof(float) * c->P, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  *bytes = need;
  return DINR_OK;
}

dinr_status dinr_set_state(dinr_ctx *c, const void *buf, size_t bytes) {
  LIVE(c);
  size_t need = sizeof(StateHeader) + 3 * sizeof(float) * c->P;
  if (!buf || bytes != need)
    return (dinr_status)dinr_fail(c, DINR_ERR_STATE, "state size mismatch");
  StateHeader h;
  memcpy(&h, buf, sizeof(h));
  if (memcmp(h.magic, "DINRST1", 8) != 0 || h.version != 1 || h.F != c->F || h.H != c->H ||
      h.W != c->W || h.P != c->P)
    return (dinr_status)dinr_fail(c, DINR_ERR_STATE, "state does not match this network");
  const float *f = (const float *)((const char *)buf + sizeof(h));
  CK(cudaMemcpyAsync(c->d_params, f, sizeof(float) * c->P, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->d_m, f + c->P, sizeof(float) * c->P, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->d_v, f + 2 * c->P, sizeof(float) * c->P, cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  c->step = h.step;
  c->sampler_seed = h.sampler_seed;
  return after_param_update(c);
}

dinr_status dinr_sample_indices(dinr_ctx *c, int64_t step, int n, int64_t *out) {
  LIVE(c);
  if (!out || n < 1 || step < 0)
    return (dinr_status)dinr_fail(c, DINR_ERR_ARG, "invalid sampler request");
  launch_sample_indices(c->n_proj, n, step, c->sampler_seed, (long long *)out, c->st);
  CKL();
  return DINR_OK;
}

// ------------------------------------------------------- phantom utility
dinr_status dinr_phantom_project(const dinr_geometry *geom, int n_ell, const double *centre,
                                 const double *axes, const double *rho, const double *vel,
                                 double growth, const int64_t *idx, int64_t n, float *out,
                                 void *cuda_stream) {
  if (!dinr_geometry_valid(geom) || n_ell < 0 || (n_ell > 0 && (!centre || !axes || !rho)) ||
      !out || n < 0)
    return (dinr_status)dinr_fail(nullptr, DINR_ERR_ARG, "invalid phantom request");
  dinr_ctx tmp;  // holds the temporary allocations and the message
  dinr_ctx *c = &tmp;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  GeoDev g{};
  double2 *cs = nullptr;
  double *tb = nullptr, *tt = nullptr;
  dinr_status s = setup_geometry(c, geom, &g, &cs, &tb, &tt, st);
  if (s == DINR_OK && n > 0) {
    std::vector<double> ell(10 * (size_t)(n_ell > 0 ? n_ell : 1), 0.0);
    for (int k = 0; k < n_ell; ++k) {
      for (int d = 0; d < 3; ++d) {
        ell[10 * k + d] = centre[3 * k + d];
        ell[10 * k + 3 + d] = axes[3 * k + d];
        ell[10 * k + 7 + d] = vel ? vel[3 * k + d] : 0.0;
      }
      ell[10 * k + 6] = rho[k];
    }
    bool ok = true;
    double *d_ell = (double *)dev_alloc(c, sizeof(double) * ell.size(), &ok);
    if (!ok) {
      s = DINR_ERR_OOM;
    } else if (cudaMemcpyAsync(d_ell, ell.data(), sizeof(double) * ell.size(),
                               cudaMemcpyHostToDevice, st) != cudaSuccess) {
      s = DINR_ERR_CUDA;
    } else {
      launch_phantom(g, tt, n_ell, d_ell, growth, (const long long *)idx, n, out, st);
      if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
        s = DINR_ERR_CUDA;
    }
  }
  if (s != DINR_OK) dinr_fail(nullptr, s, "phantom projection failed (%s)", tmp.err);
  for (void *p : tmp.allocs) cudaFree(p);
  return s;
}

// ------------------------------------------------------------ profiling
static cudaEvent_t prof_event(dinr_ctx *c) {
  if (c->prof_used == c->prof_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    c->prof_pool.push_back(e);
  }
  return c->prof_pool[c->prof_used++];
}

ProfScope::ProfScope(dinr_ctx *ctx, const char *name, double flops, double bytes) : c(ctx) {
  nvtxRangePushA(name);
  if (!c || !c->prof) return;
  int cls = -1;
  for (size_t i = 0; i < c->prof_names.size(); ++i)
    if (c->prof_names[i] == name) cls = (int)i;
  if (cls < 0) {
    c->prof_names.push_back(name);
    cls = (int)c->prof_names.size() - 1;
  }
  ProfRec r{cls, prof_event(c), prof_event(c), flops, bytes};
  if (!r.a || !r.b) return;
  cudaEventRecord(r.a, c->st);
  c->prof_recs.push_back(r);
  idx = (int)c->prof_recs.size() - 1;
}

ProfScope::~ProfScope() {
  if (idx >= 0) cudaEventRecord(c->prof_recs[idx].b, c->st);
  nvtxRangePop();
}

dinr_status dinr_profile(dinr_ctx *c, int enable) {
  LIVE(c);
  CK(cudaStreamSynchronize(c->st));
  c->prof = enable != 0;
  if (enable) {
    c->prof_recs.clear();
    c->prof_names.clear();
    c->prof_used = 0;
    c->launches = 0;
    c->samples_done = 0;
  }
  return DINR_OK;
}

dinr_status dinr_profile_report(dinr_ctx *c, char *buf, size_t size) {
  LIVE(c);
  if (!buf || size == 0) return (dinr_status)dinr_fail(c, DINR_ERR_ARG, "no buffer");
  CK(cudaStreamSynchronize(c->st));
  size_t n = c->prof_names.size();
  std::vector<double> ms(n, 0.0), fl(n, 0.0), by(n, 0.0);
  std::vector<long long> cnt(n, 0);
  for (const ProfRec &r : c->prof_recs) {
    float t = 0.0f;
    CK(cudaEventElapsedTime(&t, r.a, r.b));
    ms[r.cls] += t;
    fl[r.cls] += r.flops;
    by[r.cls] += r.bytes;
    cnt[r.cls] += 1;
  }
  std::string out;
  char line[256];
  for (size_t i = 0; i < n; ++i) {
    snprintf(line, sizeof(line), "%s %lld %.6f %.6e %.6e\n", c->prof_names[i].c_str(), cnt[i],
             ms[i], fl[i], by[i]);
    out += line;
  }
  snprintf(line, sizeof(line), "total_launches %lld 0 0 0\n", c->launches);
  out += line;
  snprintf(line, sizeof(line), "total_samples %lld 0 0 0\n", c->samples_done);
  out += line;
  snprintf(buf, size, "%s", out.c_str());
  return DINR_OK;
}
