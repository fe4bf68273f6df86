// Internal launchers of libdinr (not part of the C ABI).
#pragma once

#include "common.cuh"

namespace dinr {

// Where the samples of an encode pass come from.
enum SampleSource {
  kSrcTrainRays = 0,   // rays of projection indices (Sec. III decode)
  kSrcVirtualView = 1, // rays of a rows x cols detector at (theta, t)
  kSrcPoints = 2,      // explicit (t, z, y, x) points
  kSrcGrid = 3,        // regular grid at time t
  kSrcSubRays = 4      // samples of App. A sub-pixel rays (ragged; see subpixel.cuh)
};

struct SourceArgs {
  int kind;
  long long first;           // number of the first ray/point of this pass
  const long long *idx;      // kSrcTrainRays: ray indices (already offset)
  // kSrcVirtualView
  double vc, vs, vtbar, vpu, vpv;
  int vrows, vcols;
  // kSrcPoints
  const float *points;       // [n][4] (t, z, y, x)
  double t_scale, t_bias;    // t_bar = t * t_scale + t_bias
  // kSrcGrid
  double glo[3], gstep[3];   // (x, y, z)
  int gdims[3];              // (nx, ny, nz)
  double gtbar;
  // kSrcSubRays: sample q belongs to sub-ray owner[q], whose first sample is
  // sfirst[k]; srec (FP64) / srec32 (FP32) hold per sub-ray the normalised
  // time, the normalised first sample (z, y, x) and step (z, y, x), and l.
  const int *owner;
  const long long *sfirst;
  const double *srec;
  const float *srec32;
};

// The ray of ray slot r for each ray source kind.
__device__ __forceinline__ Ray source_ray(const GeoDev &g, const SourceArgs &s, long long r) {
  if (s.kind == kSrcTrainRays) return make_ray(g, s.idx[r]);
  long long q = s.first + r;
  int row = (int)(q / s.vcols), col = (int)(q - (long long)row * s.vcols);
  double u = g.ou + (col + 0.5) * s.vpu, v = g.ov + (row + 0.5) * s.vpv;
  return ray_at(g, u, v, s.vc, s.vs, s.vtbar);
}

// Normalised (t, z, y, x) of sample j of ray/point slot r.
__device__ __forceinline__ void source_coords(const GeoDev &g, const SourceArgs &s,
                                              long long r, int j, int S, double c[4],
                                              float *len) {
  if (s.kind == kSrcTrainRays || s.kind == kSrcVirtualView) {
    Ray ray = source_ray(g, s, r);
    c[0] = ray.tbar;
    sample_coords(g, ray, j, S, c[1], c[2], c[3]);
    *len = (float)ray.l;
  } else if (s.kind == kSrcSubRays) {
    const long long q = s.first + r;
    const int k = s.owner[q];
    const double jd = (double)(q - s.sfirst[k]);
    const double *R = s.srec + 8 * (long long)k;
    c[0] = R[0];
    c[1] = fma(jd, R[4], R[1]);
    c[2] = fma(jd, R[5], R[2]);
    c[3] = fma(jd, R[6], R[3]);
    *len = 1.0f;
  } else if (s.kind == kSrcPoints) {
    const float *p = s.points + 4 * (s.first + r);
    c[0] = (double)p[0] * s.t_scale + s.t_bias;
    c[1] = (double)p[1] * g.zs + g.zb;
    c[2] = (double)p[2] * g.inv_R;
    c[3] = (double)p[3] * g.inv_R;
    *len = 1.0f;
  } else {
    long long nx = s.gdims[0], ny = s.gdims[1], q = s.first + r;
    long long iz = q / (nx * ny), rem = q - iz * nx * ny;
    long long iy = rem / nx, ix = rem - iy * nx;
    double x = s.glo[0] + (ix + 0.5) * s.gstep[0];
    double y = s.glo[1] + (iy + 0.5) * s.gstep[1];
    double z = s.glo[2] + (iz + 0.5) * s.gstep[2];
    c[0] = s.gtbar;
    c[1] = z * g.zs + g.zb;
    c[2] = y * g.inv_R;
    c[3] = x * g.inv_R;
    *len = 1.0f;
  }
}

// Encoded features of a pass. Rays r in [0, n_rays) own samples
// [r*S, r*S + S) (S = 1 for point sources). Features are written as
// FP32 or BF16 [n_samples][ld] with zero padding from d_in to ld.
// grff_c > 0 selects the Gaussian random Fourier features of the device
// matrix grff_B [grff_c][4] in place of the octave features.
void launch_encode_f32(const GeoDev &g, const SourceArgs &src, long long n_rays, int S,
                       int F, int grff_c, const float *grff_B, int ld, float *E, float *ray_l,
                       const float *proj, float *ray_p, cudaStream_t st);
void launch_encode_bf16(const GeoDev &g, const SourceArgs &src, long long n_rays, int S,
                        int F, int grff_c, const float *grff_B, int ld, __nv_bfloat16 *E,
                        float *ray_l, const float *proj, float *ray_p, cudaStream_t st);

void launch_sample_indices(long long n_proj, int B, long long step, uint64_t seed,
                           long long *out, cudaStream_t st);
// Replaces indices outside [0, n_proj) by 0 and sets *bad.
void launch_check_indices(long long *idx, int n, long long n_proj, int *bad, cudaStream_t st);
void launch_phantom(const GeoDev &g, const double *view_t, int n_ell, const double *ell,
                    double growth, const long long *idx, long long n, float *out,
                    cudaStream_t st);

// Output layer, forward model (Eq. 1, 2) and loss terms (Eq. 3, 5).
//   zH: last hidden pre-activations (FP32 path) [n_rays*S][W] with ld;
//   writes z_out [n_samples], p_bar [n_rays], sq [n_rays] = (p_bar - p)^2 and
//   dz [n_samples] = dL/dz_out = (2/B) (p_bar - p) mu0 (l/S) out'(z_out)
//   when `train` is set (B = 1/inv_B is the whole minibatch).
void launch_out_segsum_f32(const float *zH, long long ld, int W, int act, int out_act,
                           const float *w_out, const float *b_out, long long n_rays, int S,
                           float mu0, const float *ray_l, const float *ray_p, float inv_B,
                           bool train, float *z_out, float *p_bar, float *sq, float *dz,
                           cudaStream_t st);
// Same, from per-sample outputs z_out already computed by a fused kernel.
void launch_segsum(const float *z_out, int out_act, long long n_rays, int S, float mu0,
                   const float *ray_l, const float *ray_p, float inv_B, bool train,
                   float *p_bar, float *sq, float *dz, cudaStream_t st);

// delta_H[s][c] = dz[s] * w_out[c] * act'(zH[s][c])
void launch_out_delta_f32(const float *dz, const float *w_out, const float *zH, long long ld,
                          int W, int act, long long n, float *D, cudaStream_t st);

// Column sums with split partials: part[z][c] = sum over rows of split z of
// w[s] * f(X[s][c]), f = act when apply_act, w = 1 when w == nullptr.
int colsum_splits(long long rows);
void launch_colsum(const float *X, long long ld, int C, long long rows, const float *w,
                   bool apply_act, int act, int splits, float *part, cudaStream_t st);
// out[c] = (accumulate ? out[c] : 0) + sum_z part[z][c], fixed order.
void launch_reduce_partials(const float *part, int splits, long long C, float *out,
                            bool accumulate, cudaStream_t st);
// loss = (accumulate ? loss : 0) + inv_B * sum sq[r]
void launch_loss_sum(const float *sq, long long n, float inv_B, float *loss, bool accumulate,
                     cudaStream_t st);

// Adam (Kingma & Ba), FP32 master weights.
// The sampler with its step read from device memory.
void launch_sample_indices_dev(long long n_proj, int B, const long long *step, uint64_t seed,
                               long long *out, cudaStream_t st);
// Adam with the learning rate and bias corrections of step *step from
// tab[3 (*step - *step0) ..] (lr, 1 / (1 - beta1^t), 1 / (1 - beta2^t)).
void launch_adam_tab(float *theta, float *m, float *v, const float *g, long long P, float beta1,
                     float beta2, float eps, const float *tab, const long long *step,
                     const long long *step0, cudaStream_t st);
// *step += 1 on the device.
void launch_step_inc(long long *step, cudaStream_t st);
// out = g * (*scale) over P floats (scale: device float[1]).
void launch_scale_by(const float *g, long long P, const float *scale, float *out,
                     cudaStream_t st);
void launch_adam(float *theta, float *m, float *v, const float *g, long long P, float lr,
                 float beta1, float beta2, float eps, float bc1, float bc2, cudaStream_t st);

// FP32 SIMT GEMM (the plain path). C(m, n) = sum_k A(m, k) B(n, k) with
//   A(m, k) = A[m*lda + k] (a_kc) or A[k*lda + m],
//   B(n, k) = B[n*ldb + k] (b_kc) or B[k*ldb + n],
// optional act() applied to A or B elements as loaded, and epilogues:
//   kEpiBias:    C = acc + bias[n]
//   kEpiMask:    C = acc * act'(Zp[m*ldz + n])
//   kEpiPartial: C[z] = acc over the z-th K split
enum { kEpiBias = 0, kEpiMask = 1, kEpiPartial = 2 };
struct SgemmArgs {
  int M, N;
  long long K;
  const float *A; long long lda;
  const float *B; long long ldb;
  int act;
  float *C; long long ldc;
  const float *bias;
  const float *Zp; long long ldz;
  long long k_per_split;
  long long split_stride;
};
// Returns -1 for an operand/epilogue combination that is not instantiated.
int launch_sgemm(const SgemmArgs &a, bool a_kc, bool b_kc, bool a_act, bool b_act, int epi,
                 int splits, cudaStream_t st);

}  // namespace dinr
