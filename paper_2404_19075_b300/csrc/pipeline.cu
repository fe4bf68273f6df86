// Orchestration of one training step, of re-projection and of queries.
//
// A step processes its minibatch in passes of at most chunk_rays rays. Rays
// are independent given the parameters (Eq. 1-5 couple samples only within
// a ray), so each pass runs forward, loss terms and backward on its own and
// adds its gradient into the step's gradient in a fixed order; the loss is
// normalised by the whole minibatch size (Eq. 5).
#include "context.cuh"
#include "subpixel.cuh"
#include "tc.cuh"

using namespace dinr;

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

static constexpr long long kMaxPartialFloats = 64LL << 20;

bool bf16_supported(const dinr_net *net) { return tc_supported(net); }

bool recompute_applies(const dinr_ctx *c) {
  return c->prec != DINR_PREC_FP32 && tc_recompute_applies(c);
}

long long workspace_bytes_per_sample(const dinr_ctx *c) {
  if (c->prec != DINR_PREC_FP32) return tc_bytes_per_sample(c);
  return 4LL * (c->ldE + (long long)(c->H + 2) * c->W) + 8;
}

static int dw_splits(long long rows, int M, int N) {
  int tiles = ((M + 127) / 128) * ((N + 127) / 128);
  long long s = 592 / tiles;
  long long by_rows = rows / 1024;
  if (s > by_rows) s = by_rows;
  long long by_mem = kMaxPartialFloats / ((long long)M * N);
  if (s > by_mem) s = by_mem;
  return (int)(s < 1 ? 1 : s);
}

static dinr_status f32_alloc(dinr_ctx *c);

dinr_status alloc_workspace(dinr_ctx *c) {
  dinr_status s = c->prec != DINR_PREC_FP32 ? tc_alloc(c) : f32_alloc(c);
  if (s != DINR_OK) return s;
  return subpix_alloc(c);
}

static dinr_status f32_alloc(dinr_ctx *c) {
  long long ns = (long long)c->chunk_rays * c->S;
  long long nr = ns;  // point queries use one "ray" per sample
  auto grab = [&](float **p, long long n) -> bool {
    void *q = nullptr;
    if (cudaMalloc(&q, sizeof(float) * (n > 0 ? n : 1)) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    c->allocs.push_back(q);
    *p = (float *)q;
    return true;
  };
  int maxK = c->ldE > c->W ? c->ldE : c->W;
  long long pf = (long long)dw_splits(ns, c->W, maxK) * c->W * maxK;
  long long pc = (long long)colsum_splits(ns) * c->W;
  c->part_floats = pf > pc ? pf : pc;
  bool ok = grab(&c->E, ns * c->ldE) && grab(&c->Z, ns * c->W * (long long)c->H) &&
            grab(&c->D0, ns * c->W) && grab(&c->D1, ns * c->W) && grab(&c->zout, ns) &&
            grab(&c->dz, ns) && grab(&c->ray_l, nr) && grab(&c->ray_p, nr) &&
            grab(&c->pbar, nr) && grab(&c->sq, nr) && grab(&c->part, c->part_floats);
  if (!ok) return (dinr_status)dinr_fail(c, DINR_ERR_OOM, "workspace allocation failed");
  return DINR_OK;
}

void destroy_backend(dinr_ctx *c) {
  if (c->prec != DINR_PREC_FP32) tc_destroy(c);
  subpix_free(c);
}

dinr_status backend_poll(dinr_ctx *c) {
  if (c->prec != DINR_PREC_FP32) return tc_poll(c);
  CK(cudaStreamSynchronize(c->st));
  return DINR_OK;
}

dinr_status after_param_update(dinr_ctx *c) {
  c->fwd_n = 0;  // a forward taken with the old parameters has no backward now
  c->fwd_kept = false;
  if (c->prec != DINR_PREC_FP32) return tc_params_changed(c);
  return DINR_OK;
}

// ------------------------------------------------------------ FP32 path

// Hidden layers: Z_L = act(Z_{L-1}) W_L^T + b_L (Z_{-1} = features E).
static dinr_status f32_hidden(dinr_ctx *c, long long ns) {
  for (int L = 0; L < c->H; ++L) {
    SgemmArgs a{};
    a.M = (int)ns;
    a.N = c->W;
    a.K = c->fan_in[L];
    a.A = L == 0 ? c->E : c->Z + (long long)(L - 1) * ns * c->W;
    a.lda = L == 0 ? c->ldE : c->W;
    a.B = c->d_params + c->offW[L];
    a.ldb = c->fan_in[L];
    a.act = c->act;
    a.C = c->Z + (long long)L * ns * c->W;
    a.ldc = c->W;
    a.bias = c->d_params + c->offb[L];
    a.k_per_split = a.K;
    ProfScope ps(c, "sgemm_fwd", 2.0 * ns * c->W * a.K, 4.0 * ns * (a.K + c->W));
    if (launch_sgemm(a, true, true, L > 0, false, kEpiBias, 1, c->st) != 0)
      return (dinr_status)dinr_fail(c, DINR_ERR_UNSUPPORTED, "sgemm variant");
    CKL();
  }
  return DINR_OK;
}

static float *zlast(dinr_ctx *c, long long ns) {
  return c->Z + (long long)(c->H - 1) * ns * c->W;
}

// grad[off .. off+C) (+)= column sums of X (optionally act(X), weighted by w)
static dinr_status colsum_into(dinr_ctx *c, const float *X, long long ld, int C, long long rows,
                               const float *w, bool apply_act, long long off, bool acc) {
  int splits = colsum_splits(rows);
  launch_colsum(X, ld, C, rows, w, apply_act, c->act, splits, c->part, c->st);
  CKL();
  launch_reduce_partials(c->part, splits, C, c->d_grad + off, acc, c->st);
  CKL();
  return DINR_OK;
}

// Backward of one pass (App. A gradient, chain rule by hand): output layer,
// then each hidden layer from the last: dW_L = D^T In_L, db_L = sum D, and
// D <- (D W_L) * act'(Z_{L-1}).
static dinr_status f32_backward(dinr_ctx *c, long long ns, bool acc) {
  dinr_status s;
  float *zH = zlast(c, ns);
  s = colsum_into(c, zH, c->W, c->W, ns, c->dz, true, c->offW[c->H], acc);
  if (s != DINR_OK) return s;
  s = colsum_into(c, c->dz, 1, 1, ns, nullptr, false, c->offb[c->H], acc);
  if (s != DINR_OK) return s;
  launch_out_delta_f32(c->dz, c->d_params + c->offW[c->H], zH, c->W, c->W, c->act, ns, c->D0,
                       c->st);
  CKL();
  float *D = c->D0, *Dn = c->D1;
  for (int L = c->H - 1; L >= 0; --L) {
    int K_in = c->fan_in[L];
    const float *In = L == 0 ? c->E : c->Z + (long long)(L - 1) * ns * c->W;
    long long ldIn = L == 0 ? c->ldE : c->W;
    SgemmArgs a{};
    a.M = c->W;
    a.N = K_in;
    a.K = ns;
    a.A = D;
    a.lda = c->W;
    a.B = In;
    a.ldb = ldIn;
    a.act = c->act;
    a.C = c->part;
    a.ldc = K_in;
    int splits = dw_splits(ns, c->W, K_in);
    long long cap = c->part_floats / ((long long)c->W * K_in);
    if (splits > cap) splits = (int)(cap < 1 ? 1 : cap);
    a.k_per_split = ((ns + splits - 1) / splits + 7) / 8 * 8;
    splits = (int)((ns + a.k_per_split - 1) / a.k_per_split);
    a.split_stride = (long long)c->W * K_in;
    {
      ProfScope ps(c, "sgemm_dw", 2.0 * ns * c->W * K_in, 4.0 * ns * (c->W + K_in));
      if (launch_sgemm(a, false, false, false, L > 0, kEpiPartial, splits, c->st) != 0)
        return (dinr_status)dinr_fail(c, DINR_ERR_UNSUPPORTED, "sgemm variant");
      CKL();
    }
    launch_reduce_partials(c->part, splits, (long long)c->W * K_in, c->d_grad + c->offW[L], acc,
                           c->st);
    CKL();
    s = colsum_into(c, D, c->W, c->W, ns, nullptr, false, c->offb[L], acc);
    if (s != DINR_OK) return s;
    if (L > 0) {
      SgemmArgs b{};
      b.M = (int)ns;
      b.N = c->W;
      b.K = c->W;
      b.A = D;
      b.lda = c->W;
      b.B = c->d_params + c->offW[L];
      b.ldb = c->W;
      b.act = c->act;
      b.C = Dn;
      b.ldc = c->W;
      b.Zp = c->Z + (long long)(L - 1) * ns * c->W;
      b.ldz = c->W;
      b.k_per_split = b.K;
      ProfScope ps(c, "sgemm_dx", 2.0 * ns * c->W * c->W, 4.0 * ns * 3 * c->W);
      if (launch_sgemm(b, true, false, false, false, kEpiMask, 1, c->st) != 0)
        return (dinr_status)dinr_fail(c, DINR_ERR_UNSUPPORTED, "sgemm variant");
      CKL();
      float *t = D;
      D = Dn;
      Dn = t;
    }
  }
  return DINR_OK;
}

// Per-sample outputs z_out of ns encoded samples (FP32 path).
static dinr_status f32_outputs(dinr_ctx *c, long long ns) {
  dinr_status s = f32_hidden(c, ns);
  if (s != DINR_OK) return s;
  launch_out_segsum_f32(zlast(c, ns), c->W, c->W, c->act, c->out_act,
                        c->d_params + c->offW[c->H], c->d_params + c->offb[c->H], ns, 1, c->mu0,
                        nullptr, nullptr, 1.0f, false, c->zout, nullptr, nullptr, nullptr, c->st);
  CKL();
  return DINR_OK;
}

// App. A forward model of nr pixels idx (FP32 path): sub-rays, features of
// every sample, network, ragged forward model; with train also the loss
// terms and dL/dz.
static dinr_status f32_subpix_pass(dinr_ctx *c, const long long *idx, int nr, float inv_B,
                                   bool train, float *p_bar, long long *ns_out) {
  long long ns = 0;
  dinr_status s = subpix_setup(c, idx, nr, train ? c->d_proj : nullptr, &ns);
  if (s != DINR_OK) return s;
  SourceArgs src = subpix_source(c);
  {
    ProfScope ps(c, "encode", 0.0, 4.0 * ns * c->ldE);
    launch_encode_f32(c->geo, src, ns, 1, c->F, c->grff_c, c->d_grff_B, c->ldE, c->E, nullptr,
                      nullptr, nullptr, c->st);
    CKL();
  }
  s = f32_outputs(c, ns);
  if (s != DINR_OK) return s;
  *ns_out = ns;
  return subpix_segsum(c, c->zout, nr, inv_B, train, p_bar, train ? c->sq : nullptr,
                       train ? c->dz : nullptr);
}

static dinr_status f32_loss_grad(dinr_ctx *c, int n, RunMode mode) {
  if (mode == kGradOnly) {
    dinr_status s = f32_backward(c, c->fwd_ns, false);
    c->fwd_kept = false;
    return s;
  }
  const bool one_pass = n <= c->chunk_rays;
  float inv_B = 1.0f / (float)n;
  for (int r0 = 0, pass = 0; r0 < n; r0 += c->chunk_rays, ++pass) {
    int nr = n - r0 < c->chunk_rays ? n - r0 : c->chunk_rays;
    long long ns = (long long)nr * c->S;
    if (c->geo.D > 0) {
      dinr_status s = f32_subpix_pass(c, c->d_idx + r0, nr, inv_B, true, c->pbar, &ns);
      if (s != DINR_OK) return s;
      launch_loss_sum(c->sq, nr, inv_B, c->d_loss, pass > 0, c->st);
      CKL();
      if (c->prof) c->samples_done += ns;
    } else {
      SourceArgs src{};
      src.kind = kSrcTrainRays;
      src.idx = c->d_idx + r0;
      {
        ProfScope ps(c, "encode", 0.0, 4.0 * ns * c->ldE);
        launch_encode_f32(c->geo, src, nr, c->S, c->F, c->grff_c, c->d_grff_B, c->ldE, c->E,
                          c->ray_l, c->d_proj, c->ray_p, c->st);
        CKL();
      }
      dinr_status s = f32_hidden(c, ns);
      if (s != DINR_OK) return s;
      launch_out_segsum_f32(zlast(c, ns), c->W, c->W, c->act, c->out_act,
                            c->d_params + c->offW[c->H], c->d_params + c->offb[c->H], nr, c->S,
                            c->mu0, c->ray_l, c->ray_p, inv_B, true, c->zout, c->pbar, c->sq,
                            c->dz, c->st);
      CKL();
      launch_loss_sum(c->sq, nr, inv_B, c->d_loss, pass > 0, c->st);
      CKL();
      if (c->prof) c->samples_done += ns;
    }
    if (mode == kLossOnly) {
      if (one_pass) {
        c->fwd_kept = true;
        c->fwd_ns = ns;
      }
      continue;
    }
    dinr_status s = f32_backward(c, ns, pass > 0);
    if (s != DINR_OK) return s;
  }
  return DINR_OK;
}

// Forward model of ray (S > 0) or point (S = 1, l = 1) sources, in passes.
static dinr_status f32_forward(dinr_ctx *c, const SourceArgs &src0, long long n_rays, int S,
                               float *out) {
  if (src0.kind == kSrcTrainRays && c->geo.D > 0) {  // App. A model of minibatch pixels
    for (long long r0 = 0; r0 < n_rays; r0 += c->chunk_rays) {
      int nr = (int)(n_rays - r0 < c->chunk_rays ? n_rays - r0 : c->chunk_rays);
      long long ns = 0;
      dinr_status s = f32_subpix_pass(c, src0.idx + r0, nr, 1.0f, false, out + r0, &ns);
      if (s != DINR_OK) return s;
    }
    return DINR_OK;
  }
  long long per = (long long)c->chunk_rays * c->S / S;
  if (per < 1) return (dinr_status)dinr_fail(c, DINR_ERR_ARG, "S larger than the workspace");
  for (long long r0 = 0; r0 < n_rays; r0 += per) {
    long long nr = n_rays - r0 < per ? n_rays - r0 : per;
    SourceArgs src = src0;
    if (src.kind == kSrcTrainRays)
      src.idx = src0.idx + r0;
    else
      src.first = src0.first + r0;
    long long ns = nr * S;
    launch_encode_f32(c->geo, src, nr, S, c->F, c->grff_c, c->d_grff_B, c->ldE, c->E, c->ray_l,
                      nullptr, nullptr, c->st);
    CKL();
    dinr_status s = f32_hidden(c, ns);
    if (s != DINR_OK) return s;
    launch_out_segsum_f32(zlast(c, ns), c->W, c->W, c->act, c->out_act,
                          c->d_params + c->offW[c->H], c->d_params + c->offb[c->H], nr, S,
                          c->mu0, c->ray_l, nullptr,
                          1.0f, false, c->zout, out + r0, nullptr, nullptr, c->st);
    CKL();
  }
  return DINR_OK;
}

// ------------------------------------------------------------ dispatch

dinr_status run_loss_grad(dinr_ctx *c, int n, RunMode mode) {
  if (mode != kGradOnly) c->fwd_kept = false;
  if (c->prec != DINR_PREC_FP32) return tc_loss_grad(c, n, mode);
  return f32_loss_grad(c, n, mode);
}

dinr_status run_forward_rays(dinr_ctx *c, const SourceArgs &src, long long n_rays, int S,
                             float *out) {
  c->fwd_kept = false;
  if (c->prec != DINR_PREC_FP32) return tc_forward_rays(c, src, n_rays, S, out);
  return f32_forward(c, src, n_rays, S, out);
}

dinr_status run_forward_points(dinr_ctx *c, const SourceArgs &src, long long n, float *out) {
  c->fwd_kept = false;
  if (c->prec != DINR_PREC_FP32) return tc_forward_points(c, src, n, out);
  return f32_forward(c, src, n, 1, out);
}
