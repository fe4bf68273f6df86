/*
 * dinr.h - C ABI of libdinr, a single-GPU (sm_103a) implementation of the
 * stochastic training step of DINR (distributed implicit neural
 * representation) for 4D time-space CT reconstruction, and of the queries
 * served by a trained network.
 *
 * Method (paper sections cited per entry point):
 *   Sec. III    projection index i = m*N + n, view m at angle theta_m and
 *               time T_m; rotating the object by theta equals rotating the
 *               source/detector pair by -theta.
 *   Eq. 1, 2    forward model p_bar_i = (1/|Phi_i|) sum_j w(r_ij) M(r_ij),
 *               w = mu0 * l (l: length of the ray inside the cylindrical FOV).
 *   Eq. 3, 5    squared error d_i and minibatch loss L = mean over Omega of d_i.
 *   App. A      ray sampling (equispaced samples on the FOV chord) and the
 *               gradient of L with respect to the network parameters.
 *   App. B      network: normalise (t,z,y,x) to [-1,1], Fourier features,
 *               fully connected hidden layers, linear output.
 *   Sec. III,
 *   App. C      Adam, learning rate 1e-3, optional decay per epoch.
 *
 * Conventions for every call:
 *   - Status codes are returned, never abort(). A CUDA error makes the
 *     context sticky-failed: later calls return DINR_ERR_CUDA.
 *     dinr_last_error() gives a message for the last failure.
 *   - All device work is enqueued on the context's stream (given at
 *     creation; NULL = the legacy default stream). Calls return without
 *     waiting unless they write a host output.
 *   - Host arrays passed in are copied before the call returns. Device
 *     arrays passed in are borrowed for the stream-ordered duration of the
 *     call: they must stay valid until the stream reaches that point.
 *   - The flat parameter vector (FP32) is laid out as
 *       [W_1 (width x d_in, row-major), b_1 (width),
 *        W_2 (width x width), b_2, ..., W_H, b_H, w_out (width), b_out (1)]
 *     with d_in = 4 + 8 * n_freq (octave encoding) or 2 * grff_c (GRFF);
 *     its length is dinr_param_count() / dinr_param_count_din().
 *   - Features of a normalised coordinate r = (t,z,y,x) are, with the octave
 *     encoding, [t, z, y, x, then for c in (t,z,y,x), l = 0..F-1:
 *     sin(2^l pi c), cos(2^l pi c)]; with the Gaussian random Fourier
 *     features of App. B item 2, [cos(2 pi B r) (C values), sin(2 pi B r)
 *     (C values)] for the frozen C x 4 matrix B.
 *   - Pixel centres: u = det_off_u + (col + 0.5) * det_pitch_u,
 *     v = det_off_v + (row + 0.5) * det_pitch_v; detector rows run along +z.
 *     At theta = 0 rays travel along +y and u runs along +x; the cone-beam
 *     source is at (0, -sod, 0) and the detector plane at distance sdd from
 *     it. Each pixel has one ray through its centre; a ray carries
 *     samples_per_ray samples at the midpoints of equal sub-intervals of its
 *     chord through the FOV cylinder x^2 + y^2 <= fov_r^2,
 *     fov_z0 <= z <= fov_z1. A ray that misses the FOV predicts 0.
 */
#ifndef DINR_H
#define DINR_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define DINR_API __attribute__((visibility("default")))
#else
#define DINR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DINR_OK = 0,
  DINR_ERR_ARG = 1,          /* invalid argument (null pointer, bad size, ...) */
  DINR_ERR_OOM = 2,          /* device or host allocation failed */
  DINR_ERR_CUDA = 3,         /* a CUDA call failed; the context is now unusable */
  DINR_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up */
  DINR_ERR_NONFINITE = 5,    /* the loss of a step was NaN or infinite */
  DINR_ERR_UNSUPPORTED = 6,  /* the shape or mode is not supported by the library */
  DINR_ERR_BUSY = 7,         /* the request cannot be admitted now */
  DINR_ERR_STATE = 8         /* the call is out of order or the state blob is bad */
} dinr_status;

enum { DINR_BEAM_PARALLEL = 0, DINR_BEAM_CONE = 1 };
enum { DINR_ACT_RELU = 0, DINR_ACT_SWISH = 1 };
enum { DINR_OUT_IDENTITY = 0, DINR_OUT_SOFTPLUS = 1 };
enum { DINR_ENC_OCTAVE = 0, DINR_ENC_GRFF = 1 };
/* Arithmetic of the network GEMMs. Geometry, segment sums, loss and the
 * Adam master weights are FP32 (ray geometry FP64) in every mode.
 *   FP32: SIMT FP32 GEMMs, activations kept in HBM (the plain path).
 *   BF16: tcgen05 tensor-core GEMMs, BF16 operands, FP32 accumulation.
 *   FP8:  measured variant: the forward GEMMs take E4M3 operands with
 *         per-tensor scales (weights: amax / 448 after every update;
 *         features: 1; hidden outputs: delayed scaling, the amax of the
 *         previous training step / 448, 1/32 before the first step;
 *         forward-only calls use the current scales and do not update
 *         them) and FP32 accumulation; the backward is the BF16 one, run on
 *         the BF16 copies of the same activations. Unfused GEMMs only (no
 *         fused chains, no recomputation; the query server runs its
 *         requests through the single-query path). */
enum { DINR_PREC_FP32 = 0, DINR_PREC_BF16 = 1, DINR_PREC_FP8 = 2 };

typedef struct dinr_ctx dinr_ctx;

/* Acquisition geometry (Sec. III, App. A), object units. */
typedef struct {
  int beam;                      /* DINR_BEAM_PARALLEL or DINR_BEAM_CONE */
  int n_views;                   /* M */
  int det_rows, det_cols;        /* N = det_rows * det_cols pixels per view */
  const double *view_angle;      /* host [n_views]: theta_m in radians; copied */
  const double *view_time;       /* host [n_views]: T_m in [t0, t1]; copied */
  double det_pitch_u, det_pitch_v;
  double det_off_u, det_off_v;
  double sod, sdd;               /* cone beam only: source-axis, source-detector */
  double fov_r, fov_z0, fov_z1;  /* cylindrical field of view */
  double t0, t1;                 /* time range used for normalisation */
  int samples_per_ray;           /* S, 1..4096 */
  double mu0;                    /* Eq. 2 scale, about the mean attenuation */
  int subpixels;                 /* forward model of training and prediction:
                                    0 (or 1 with the fixed S): one ray through
                                    each pixel centre, samples_per_ray samples;
                                    D >= 1: App. A: D x D rays to the centres
                                    of the pixel's sub-pixels, each sampled at
                                    the midpoints of ceil(l / spacing) equal
                                    parts of its chord l, spacing = pixel pitch
                                    back-projected through the rotation axis
                                    (x SOD/SDD for a cone beam) / D, and
                                    p_bar = (1/|Phi|) sum mu0 l M over all the
                                    pixel's samples (|Phi| samples). 0..8 */
} dinr_geometry;

/* Network shape (App. B). */
typedef struct {
  int n_freq;                    /* F octaves per coordinate, 0..16 */
  int hidden_layers;             /* H, 1..32 */
  int width;                     /* W; FP32 path: 1..1024; BF16 path: see
                                    DINR_ERR_UNSUPPORTED from dinr_create */
  int act;                       /* DINR_ACT_* for hidden layers */
  int out_act;                   /* DINR_OUT_* for the output */
  int prec;                      /* DINR_PREC_* */
  const float *init_params;      /* host [dinr_param_count]; copied. NULL: He
                                    initialisation from `seed` */
  uint64_t seed;
  int encoding;                  /* DINR_ENC_OCTAVE (n_freq used) or
                                    DINR_ENC_GRFF (grff_c, grff_B used) */
  int grff_c;                    /* C, even, 2..128 */
  const float *grff_B;           /* host [grff_c][4], columns (t, z, y, x);
                                    frozen; copied (App. B item 2: column t
                                    ~ N(0, sigma_t^2), z y x ~ N(0, sigma_s^2)) */
} dinr_net;

/* Optimiser and minibatch (Sec. III, App. C). */
typedef struct {
  double lr, beta1, beta2, eps;  /* Adam; 0 selects 1e-3, 0.9, 0.999, 1e-8 */
  double lr_decay_per_epoch;     /* lr *= this after each epoch; 0 selects 1 */
  int batch_rays;                /* largest minibatch |Omega| a step may use */
  int chunk_rays;                /* rays processed per pass inside a step
                                    (bounds activation memory); 0 = automatic */
  uint64_t sampler_seed;
  int recompute;                 /* activation recomputation of the BF16 path
                                    without fused chains (W > 256): 0 keeps
                                    every hidden output of a pass; 1 keeps
                                    h_L for L % k == k - 1 (k = ceil(sqrt(H)))
                                    and the last layer, and recomputes the
                                    others in the backward with the same GEMM
                                    (bitwise equal gradients, about 1/2 of a
                                    forward more work, fewer activation bytes
                                    per sample, so larger passes); negative:
                                    on when a whole minibatch does not fit in
                                    one pass without it. Ignored elsewhere. */
} dinr_train;

/* Number of FP32 parameters of a network shape (-1 for an invalid shape). */
DINR_API int64_t dinr_param_count(int n_freq, int hidden_layers, int width);
/* The same for any encoding width d_in (2 * grff_c for GRFF); -1 on bad
 * arguments. */
DINR_API int64_t dinr_param_count_din(int d_in, int hidden_layers, int width);

/* Create a context: copies geometry, parameters and the measured projection
 * stack p[M*N] (FP32, index i = m*N + n, Sec. III) to the device, zeroes the
 * Adam moments and allocates the workspace for train.batch_rays rays.
 *   proj_on_device: 0 if proj is a host pointer, 1 if a device pointer.
 *   cuda_stream: a cudaStream_t (NULL for the default stream).
 * Errors: DINR_ERR_ARG for invalid shapes or pointers, DINR_ERR_UNSUPPORTED
 * for shapes the selected precision cannot run, DINR_ERR_OOM, DINR_ERR_CUDA.
 * On failure *out is NULL. */
DINR_API dinr_status dinr_create(const dinr_geometry *geom, const dinr_net *net,
                        const dinr_train *train, const float *proj,
                        int proj_on_device, void *cuda_stream, dinr_ctx **out);

/* Replace the measured projection stack (same size as at creation). */
DINR_API dinr_status dinr_set_projections(dinr_ctx *ctx, const float *proj, int on_device);

/* One stochastic training step (Sec. III, Fig. 1(d) on one process): ray
 * generation at each sampled pixel's view angle and time, S samples per ray,
 * Fourier encoding, MLP, forward model (Eq. 1, 2), loss (Eq. 5), gradient
 * (App. A) and one Adam update of the parameters.
 *   ray_idx: n projection indices in [0, M*N) (int64), host or device per
 *            idx_on_device; NULL draws the minibatch with the built-in
 *            sampler (see dinr_sample_indices).
 *   n:       1..train.batch_rays.
 *   loss_out: host pointer that receives L; the call then waits for the
 *            step. NULL: no wait, the loss stays on the device.
 * Host indices are read before the call returns (pinned memory included:
 * with loss_out the call waits; without it, it waits for their copy).
 * With host indices and loss_out (and neither the App. A forward model
 * nor profiling) the step runs as one launch of a CUDA graph of the step,
 * captured at the first such call for each n on a private stream and
 * ordered after and before the context stream's work by events; the
 * result is bitwise that of the ordinary launches.
 * Errors: DINR_ERR_ARG (n out of range; a host index outside [0, M*N); a
 * device index outside it is replaced by 0 and reported when the call
 * waits), DINR_ERR_NONFINITE (loss_out given and L is not finite; the
 * parameters are still updated), DINR_ERR_CUDA. */
DINR_API dinr_status dinr_train_step(dinr_ctx *ctx, const int64_t *ray_idx, int n,
                            int idx_on_device, float *loss_out);

/* `steps` training steps of n rays each from the built-in sampler, as that
 * many dinr_train_step(ctx, NULL, n, 0, ...) calls would run them (the
 * same minibatches, learning rates of App. C and Adam bias corrections;
 * bitwise the same parameters), replayed from a CUDA graph of one step:
 * the first call for a given n captures the step on a private stream
 * (the sampler and Adam read the step counter and a table of per-step
 * learning rates and bias corrections from device memory), later calls
 * replay it, ordered after and before the context stream's work by
 * events. loss_out: host float, the last step's loss (the call then waits
 * for it), or NULL (no wait). Steps of the App. A forward model (which
 * read each pass's sample count back) and steps while profiling is on run
 * as ordinary steps. Errors as dinr_train_step. */
DINR_API dinr_status dinr_train_graph(dinr_ctx *ctx, int n, int steps, float *loss_out);

/* Loss and gradient only (no Adam update), for a caller-owned optimiser or an
 * autograd wrapper. loss_dev: device float[1]; grad_dev: device
 * float[dinr_param_count]. Either may be NULL. Indices as in
 * dinr_train_step. */
DINR_API dinr_status dinr_loss_grad(dinr_ctx *ctx, const int64_t *ray_idx, int n,
                           int idx_on_device, float *loss_dev, float *grad_dev);

/* dinr_loss_grad in two halves, for an autograd function whose backward
 * runs only when a gradient is asked for (Eq. 1-5 forward; App. A
 * gradient "partiald" backward).
 * dinr_forward: stages the minibatch (indices as in dinr_train_step), runs
 * the forward model and the loss (Eq. 5) and writes L to loss_dev (device
 * float[1], or NULL). It launches no backward kernel. When the minibatch is
 * one pass of the workspace (n <= chunk_rays), the activations the backward
 * needs stay in the workspace; otherwise only the loss is kept.
 * dinr_backward: the gradient of dloss * L for the minibatch of the last
 * dinr_forward, into the context's gradient (dinr_get_grads) and, when
 * grad_dev is not NULL, device float[dinr_param_count]. dloss_dev: device
 * float[1] (the upstream factor), or NULL for 1. It runs the adjoint
 * kernels on the kept activations, or, when none were kept (several
 * passes, or the workspace was used since), the whole step again with the
 * same indices and parameters (the same result).
 * Errors: DINR_ERR_ARG from dinr_backward when there is no minibatch to
 * differentiate: no dinr_forward yet, or since it another call restaged
 * indices (train_step, loss_grad, predict) or changed the parameters
 * (set_params, set_state, an Adam step). Asynchronous on the context
 * stream; errors otherwise as dinr_loss_grad. */
DINR_API dinr_status dinr_forward(dinr_ctx *ctx, const int64_t *ray_idx, int n,
                                  int idx_on_device, float *loss_dev);
DINR_API dinr_status dinr_backward(dinr_ctx *ctx, const float *dloss_dev, float *grad_dev);

/* Forward model only (Eq. 1, 2): p_bar for n rays into device float[n]. */
DINR_API dinr_status dinr_predict(dinr_ctx *ctx, const int64_t *ray_idx, int n,
                         int idx_on_device, float *pbar_dev);

/* Re-projection of the network (Eq. 1, 2) at an arbitrary angle theta and
 * time t on a rows x cols detector that covers the same physical area as
 * the acquisition detector, with S samples per ray. out_dev: device
 * float[rows*cols], row-major. rows*cols*S <= 2^31. */
DINR_API dinr_status dinr_project(dinr_ctx *ctx, double theta, double t, int rows,
                         int cols, int S, float *out_dev);

/* Reconstructed attenuation mu0 * M(r) (App. B item 4; Sec. V inference) at
 * n coordinates. coords_dev: device float[n][4] ordered (t, z, y, x) in
 * object units; out_dev: device float[n]. */
DINR_API dinr_status dinr_query(dinr_ctx *ctx, const float *coords_dev, int64_t n,
                       float *out_dev);

/* mu0 * M on a regular grid at time t (Sec. V): voxel (k, j, i) (z, y, x
 * order, x fastest) sits at lo + (index + 0.5) * (hi - lo) / dims.
 * lo, hi: host double[3] as (x, y, z); dims: host int[3] as (nx, ny, nz).
 * out_dev: device float[nz*ny*nx]. A time slice is nz = 1. */
DINR_API dinr_status dinr_query_grid(dinr_ctx *ctx, double t, const double *lo,
                            const double *hi, const int *dims, float *out_dev);

/* 4D export (Sec. V: the reconstruction at every view time). For each
 * times[k] the grid of dinr_query_grid (lo, hi, dims as there) is computed
 * and copied to pinned host memory while the next volume is computed; then
 * sink(user, k, times[k], volume, n) is called on the calling thread, in
 * order k = 0, 1, ..., with volume valid until the sink returns (host
 * float[nz*ny*nx], x fastest). A nonzero return from the sink stops the
 * export (DINR_ERR_STATE). Uses two device and two pinned host volumes of
 * 4 * nx * ny * nz bytes for the duration of the call. Synchronous. */
typedef int (*dinr_volume_sink)(void *user, int k, double t, const float *volume, int64_t n);
DINR_API dinr_status dinr_export(dinr_ctx *ctx, const double *times, int n_times,
                                 const double *lo, const double *hi, const int *dims,
                                 dinr_volume_sink sink, void *user);

/* ----------------------------------------------------------------------
 * Query server (Sec. V: inference from the trained network). Requests of
 * different kinds and sizes are batched continuously: each dinr_serve_step
 * runs one persistent launch over work taken from the in-flight requests
 * in the order of the scheduling policy (whole 128-sample tiles, whole
 * rays), so large requests span several launches and requests that arrive
 * in the meantime join the next one. Weights and per-request work lists
 * stay on the device. Contexts whose network the fused chain does not take
 * (FP32, FP8, BF16 widths above 256) are served with the same admission and
 * scheduling, the pieces of a batch running one after another through the
 * single-query path (bitwise the results of the single-query calls).
 * ---------------------------------------------------------------------- */
enum { DINR_QUERY_POINTS = 0, DINR_QUERY_GRID = 1, DINR_QUERY_PROJECT = 2 };
typedef struct {
  int kind;                      /* DINR_QUERY_* */
  const float *coords_dev;       /* POINTS: device float[n][4] (t, z, y, x) */
  int64_t n;                     /* POINTS: number of points */
  double t;                      /* GRID, PROJECT: time */
  double lo[3], hi[3];           /* GRID: box (x, y, z), as dinr_query_grid */
  int dims[3];                   /* GRID: (nx, ny, nz) */
  double theta;                  /* PROJECT: angle */
  int rows, cols, S;             /* PROJECT: detector and samples per ray */
  float *out_dev;                /* device output, caller-owned: mu0*M per point /
                                    voxel (z, y, x order) or p_bar per pixel
                                    (row-major); valid once the request is done */
} dinr_request;

/* Batch size (samples per launch, rounded down to whole 128-sample tiles,
 * at most the context's workspace) and the admission budget: requests are
 * admitted while the outputs of in-flight requests fit max_inflight_bytes.
 * 0 keeps the current value (defaults: the workspace; 4 GiB). */
DINR_API dinr_status dinr_serve_config(dinr_ctx *ctx, int64_t max_batch_samples,
                                       int64_t max_inflight_bytes);
/* Scheduling policy of the batches. DINR_SERVE_ARRIVAL (the default): work
 * is taken from requests in arrival order, which keeps the worst latency
 * lowest when the server is overloaded. DINR_SERVE_LEAST_WORK: from the
 * requests with the least work left first, so small requests do not queue
 * behind large ones (lower median latency); a request passed over for 16
 * batches in a row goes first. Results do not depend on the policy.
 * DINR_ERR_ARG for an unknown policy. */
enum { DINR_SERVE_ARRIVAL = 0, DINR_SERVE_LEAST_WORK = 1 };
DINR_API dinr_status dinr_serve_policy(dinr_ctx *ctx, int policy);
/* Admit a request. *id receives its handle. DINR_ERR_BUSY: the in-flight
 * budget is full (nothing was admitted; retry after requests complete).
 * The request's input and output memory must stay valid until it is done. */
DINR_API dinr_status dinr_serve_submit(dinr_ctx *ctx, const dinr_request *req, int64_t *id);
/* Launch one batch (no wait). *in_flight receives the number of admitted
 * requests not yet complete. */
DINR_API dinr_status dinr_serve_step(dinr_ctx *ctx, int *in_flight);
/* *done = 1 once request id has completed on the GPU (reported once). */
DINR_API dinr_status dinr_serve_poll(dinr_ctx *ctx, int64_t id, int *done);

/* Copy parameters in or out (FP32, flat layout above); on_device selects
 * whether the caller's pointer is a device pointer. Setting parameters does
 * not reset the Adam moments. */
DINR_API dinr_status dinr_set_params(dinr_ctx *ctx, const float *params, int on_device);
DINR_API dinr_status dinr_get_params(dinr_ctx *ctx, float *params, int on_device);

/* The FP32 gradient of the last dinr_train_step / dinr_loss_grad, to host. */
DINR_API dinr_status dinr_get_grads(dinr_ctx *ctx, float *host);

/* The loss of the last step (host float), waiting for it. */
DINR_API dinr_status dinr_get_loss(dinr_ctx *ctx, float *host);

/* Checkpoint: parameters, Adam m and v, step counter and sampler seed as
 * one opaque blob. With buf == NULL, *bytes receives the size.
 * dinr_set_state checks size and shape (DINR_ERR_STATE). */
DINR_API dinr_status dinr_get_state(dinr_ctx *ctx, void *buf, size_t *bytes);
DINR_API dinr_status dinr_set_state(dinr_ctx *ctx, const void *buf, size_t bytes);

/* The minibatch the built-in sampler draws at training step `step`
 * (0-based; Sec. III: random pixel subsets, an epoch is ceil(MN/n) steps):
 * slot b of step s in epoch e = s div ceil(MN/n) takes
 * pi_e(((s mod ceil(MN/n)) * n + b) mod MN), where pi_e is a 4-round
 * Feistel bijection keyed by SplitMix64 outputs 4e..4e+3 of sampler_seed,
 * restricted to [0, MN) by cycle walking. out_dev: device int64[n]. */
DINR_API dinr_status dinr_sample_indices(dinr_ctx *ctx, int64_t step, int n, int64_t *out_dev);

/* Context-free utility: exact line integrals over the FOV chord (Sec. III:
 * only the FOV contributes) of an ellipsoid phantom, sum over k of
 * rho_k * |chord of ellipsoid k| with centre c_k + vel_k * t and semi-axes
 * a_k * (1 + growth * t), each ray at its view's time, for n projection
 * indices (device int64, or NULL for all M*N in order). The phantom arrays
 * are host double[n_ell*3] as (x,y,z) and double[n_ell]; vel may be NULL.
 * out_dev: device float[n]. Used to synthesise measurements. */
DINR_API dinr_status dinr_phantom_project(const dinr_geometry *geom, int n_ell,
                                 const double *centre, const double *axes,
                                 const double *rho, const double *vel,
                                 double growth, const int64_t *idx_dev,
                                 int64_t n, float *out_dev, void *cuda_stream);

/* The projection of dinr_phantom_project, for callers that cannot allocate
 * device memory. dinr_phantom_project stages its geometry table and
 * ellipsoid parameters in device memory it allocates on every call; some
 * callers must not do that, for example a host application whose device
 * memory is owned by its own pool allocator under a fixed budget, or a
 * latency-bound loop that cannot afford cudaMalloc/cudaFree and the device
 * synchronisation that cudaFree implies. This variant stages the same data in
 * one static device array instead and calls no cudaMalloc, cudaFree or any
 * other allocating routine. The paper has no counterpart: it is a property
 * of this library, not of the method.
 *   Limits: n_views <= 4096 and n_ell <= 1024, otherwise DINR_ERR_ARG. The
 *   array (208 KiB) lives on every GPU that loads the library until the
 *   process exits.
 *   The first call on a device looks the array's device address up (with
 *   that device current) and caches it for the device's context; make that
 *   first call before any stream capture. If the device's context changes
 *   (after cudaDeviceReset, say), the next call looks the address up again.
 *   All calls on a device share the array, which keeps the last call's
 *   contents: calls whose work overlaps on the GPU (for example on two
 *   streams at once) race and give wrong results; serialise them.
 *   The host arrays (geometry tables, centre, axes, rho, vel) are read only
 *   during the call: the view table and ellipsoid records are built from
 *   them in a static host buffer and copied from there, so the caller may
 *   change or free them once the call returns.
 *   Arguments, output and errors as dinr_phantom_project (the same geometry
 *   checks), except that the call does not wait for the stream: out_dev is
 *   ready when the stream reaches the end of the call's work. */
DINR_API dinr_status dinr_phantom_project_noalloc(const dinr_geometry *geom, int n_ell,
                                                  const double *centre, const double *axes,
                                                  const double *rho, const double *vel,
                                                  double growth, const int64_t *idx_dev,
                                                  int64_t n, float *out_dev, void *cuda_stream);

/* Per-kernel timing of the context's own launches with CUDA events on its
 * stream (tracing; no counterpart in the paper). dinr_profile(ctx, 1)
 * clears and starts recording, 0 stops. dinr_profile_report waits for the
 * stream and writes one line per kernel class,
 *   "<name> <launches> <total_ms> <flops> <bytes>\n"
 * (flops and bytes: algorithmic totals over the recorded launches), then
 * "total_launches <n> 0 0 0" counting every kernel the context launched
 * since profiling started, into buf of size `size` (truncated,
 * NUL-terminated). */
DINR_API dinr_status dinr_profile(dinr_ctx *ctx, int enable);
DINR_API dinr_status dinr_profile_report(dinr_ctx *ctx, char *buf, size_t size);

/* Wait for all work of the context. */
DINR_API dinr_status dinr_synchronize(dinr_ctx *ctx);

/* Diagnostics: exercises the bounded waits of the tensor-core kernels
 * without any fault. One warp waits on a barrier that nothing arrives on,
 * through the same wait primitive and error-flag protocol as the persistent
 * kernels but with a limit of limit_ns (1 ms .. 4 s) instead of 4 s; the
 * kernel gives up, records the timeout and returns, and the call returns
 * DINR_ERR_TIMEOUT as a real timeout would. The context stays usable. */
DINR_API dinr_status dinr_selftest_timeout(dinr_ctx *ctx, int64_t limit_ns);

/* Message of the last failure of this context (or of the last failed
 * creation when ctx is NULL). Never NULL. */
DINR_API const char *dinr_last_error(const dinr_ctx *ctx);

/* Free everything the context owns. Safe on NULL. */
DINR_API void dinr_destroy(dinr_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* DINR_H */
