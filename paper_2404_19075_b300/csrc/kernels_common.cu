// Non-GEMM kernels of libdinr: minibatch sampler, phantom projector, ray
// generation + Fourier encoding, output layer + forward model + loss,
// column sums, ordered reductions and Adam.
#include "internal.cuh"

namespace dinr {

// ----------------------------------------------------------------- sampler
// Keyed Feistel bijection of [0, 2^(2h)) with cycle walking into [0, n)
// (Sec. III draws random pixel subsets; this is the library's construction).
__device__ __forceinline__ uint64_t feistel(uint64_t x, const uint64_t *key, int h) {
  uint64_t mask = (1ULL << h) - 1ULL;
  uint64_t L = x >> h, R = x & mask;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    uint64_t nl = R;
    R = L ^ (mix64(R ^ key[r]) & mask);
    L = nl;
  }
  return (L << h) | R;
}

__device__ __forceinline__ long long sample_index(long long n, int B, long long step,
                                                  uint64_t seed, int h, int b) {
  long long spe = (n + B - 1) / B;
  long long e = step / spe, j = step - e * spe;
  uint64_t key[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) key[r] = mix64(seed + (uint64_t)(4 * e + r + 1) * kGamma);
  uint64_t x = (uint64_t)((j * (long long)B + b) % n);
  uint64_t y = feistel(x, key, h);
  // Cycle walking ends: x < n lies on the cycle of a bijection.
  while (y >= (uint64_t)n) y = feistel(y, key, h);
  return (long long)y;
}

__global__ void k_sample(long long n, int B, long long step, uint64_t seed, int h,
                         long long *out) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) out[b] = sample_index(n, B, step, seed, h, b);
}

// The same with the step read from device memory (graph-replayed steps).
__global__ void k_sample_dev(long long n, int B, const long long *step, uint64_t seed, int h,
                             long long *out) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) out[b] = sample_index(n, B, *step, seed, h, b);
}

static int sampler_half_bits(long long n) {
  int bits = 2;
  while ((1LL << bits) < n) ++bits;
  return (bits + 1) / 2;
}

void launch_sample_indices(long long n, int B, long long step, uint64_t seed, long long *out,
                           cudaStream_t st) {
  k_sample<<<ceil_div(B, 256), 256, 0, st>>>(n, B, step, seed, sampler_half_bits(n), out);
}

void launch_sample_indices_dev(long long n, int B, const long long *step, uint64_t seed,
                               long long *out, cudaStream_t st) {
  k_sample_dev<<<ceil_div(B, 256), 256, 0, st>>>(n, B, step, seed, sampler_half_bits(n), out);
}

__global__ void k_check_indices(long long *idx, int n, long long n_proj, int *bad) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && (idx[i] < 0 || idx[i] >= n_proj)) {
    idx[i] = 0;
    atomicExch(bad, 1);
  }
}
void launch_check_indices(long long *idx, int n, long long n_proj, int *bad, cudaStream_t st) {
  k_check_indices<<<ceil_div(n, 256), 256, 0, st>>>(idx, n, n_proj, bad);
}

// ----------------------------------------------------------------- phantom
// ell: per ellipsoid 10 doubles: centre(3), axes(3), rho, vel(3).
__global__ void k_phantom(GeoDev g, const double *view_t, int n_ell, const double *ell,
                          double growth, const long long *idx, long long n, float *out) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= n) return;
  long long i = idx ? idx[q] : q;
  if (i < 0 || i >= g.n_proj) {
    out[q] = 0.0f;
    return;
  }
  Ray r = make_ray(g, i);
  double t = view_t[i / g.n_pixels];
  double s1 = r.s0 + r.l, acc = 0.0;
  if (r.l > 0.0) {
    for (int k = 0; k < n_ell; ++k) {
      const double *e = ell + 10 * k;
      double f = 1.0 + growth * t;
      double qx = (r.ox - e[0] - e[7] * t) / (e[3] * f);
      double qy = (r.oy - e[1] - e[8] * t) / (e[4] * f);
      double qz = (r.oz - e[2] - e[9] * t) / (e[5] * f);
      double rx = r.dx / (e[3] * f), ry = r.dy / (e[4] * f), rz = r.dz / (e[5] * f);
      double A = rx * rx + ry * ry + rz * rz;
      double B = 2.0 * (qx * rx + qy * ry + qz * rz);
      double C = qx * qx + qy * qy + qz * qz - 1.0;
      double disc = B * B - 4.0 * A * C;
      if (disc <= 0.0) continue;
      double sq = sqrt(disc);
      double lo = fmax((-B - sq) / (2.0 * A), r.s0);
      double hi = fmin((-B + sq) / (2.0 * A), s1);
      if (hi > lo) acc += e[6] * (hi - lo);
    }
  }
  out[q] = (float)acc;
}

void launch_phantom(const GeoDev &g, const double *view_t, int n_ell, const double *ell,
                    double growth, const long long *idx, long long n, float *out,
                    cudaStream_t st) {
  k_phantom<<<ceil_div(n, 128), 128, 0, st>>>(g, view_t, n_ell, ell, growth, idx, n, out);
}

// ---------------------------------------------------- rays and encoding
// Features of one coordinate at octaves 0..F-1 into sc[2F] (sin, cos).
// kFast (BF16 path): exact sincospif at octaves 0, 4, 8, ..., and angle
// doubling in between (sin 2a = 2 sin a cos a, cos 2a = (cos a - sin a)
// (cos a + sin a)); three doublings grow the error to about 1e-6, far below
// BF16 resolution. Otherwise every octave uses the exact reduction.
template <bool kFast>
__device__ __forceinline__ void coord_features(double c, int F, float *sc) {
  if (!kFast) {
    octave_features(c, F, sc);
    return;
  }
  float hi = (float)c;
  float lo = (float)(c - (double)hi);
  float scale = 1.0f, sp = 0.0f, cp = 1.0f;
  for (int l = 0; l < F; ++l) {
    if ((l & 3) == 0) {
      float a = hi * scale;
      float n = 2.0f * rintf(0.5f * a);
      float y = (a - n) + lo * scale;
      sincospif(y, &sp, &cp);
    } else {
      float s2 = 2.0f * sp * cp;
      cp = (cp - sp) * (cp + sp);
      sp = s2;
    }
    sc[2 * l] = sp;
    sc[2 * l + 1] = cp;
    scale *= 2.0f;
  }
}

template <typename T>
struct FeatWriter;
// FP32 rows: one 32-bit word per feature.
template <>
struct FeatWriter<float> {
  static constexpr int kPerWord = 1;
  __device__ static void put(uint32_t *row, int f, float a, float b) {
    row[f] = __float_as_uint(a);
    row[f + 1] = __float_as_uint(b);
  }
};
// BF16 rows: one 32-bit word per pair of adjacent features.
template <>
struct FeatWriter<__nv_bfloat16> {
  static constexpr int kPerWord = 2;
  __device__ static void put(uint32_t *row, int f, float a, float b) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    row[f >> 1] = *reinterpret_cast<uint32_t *>(&v);
  }
};

constexpr int kEncThreads = 128;

// One block encodes kEncThreads consecutive samples. The rays they belong
// to are set up once each (FP64) into shared memory, together with the
// time features of the ray (constant along it); each thread then forms its
// sample's row of features in shared memory, and the block writes its rows,
// which are contiguous in E, with coalesced 32-bit stores. ray_l receives
// each ray's chord length (1 for point sources, so that the forward model
// reduces to mu0 * M); ray_p the measured value of each training ray.
// Gaussian random Fourier features (App. B item 2) of one sample: for
// frequency k, u = B[k] . r; cos(2 pi u) into column k, sin(2 pi u) into
// column C + k. The phase is reduced exactly, 2u - 2 rint(u) in [-1, 1], then
// sincospif; u is formed in FP64 for the FP32 path and in FP32 (error about
// 1e-7 |u|, far below BF16 resolution) for the BF16 path.
template <typename T, bool kFast>
__device__ __forceinline__ void grff_row(uint32_t *row, const double (&c)[4], const float *B,
                                         int C) {
  for (int k = 0; k < C; k += 2) {
    float sv[2], cv[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const float *b = B + 4 * (k + e);
      float y;
      if (kFast) {
        const float u = fmaf(b[0], (float)c[0],
                             fmaf(b[1], (float)c[1], fmaf(b[2], (float)c[2], b[3] * (float)c[3])));
        y = 2.0f * (u - rintf(u));
      } else {
        const double u = (double)b[0] * c[0] + (double)b[1] * c[1] + (double)b[2] * c[2] +
                         (double)b[3] * c[3];
        y = (float)(2.0 * (u - rint(u)));
      }
      sincospif(y, &sv[e], &cv[e]);
    }
    FeatWriter<T>::put(row, k, cv[0], cv[1]);
    FeatWriter<T>::put(row, C + k, sv[0], sv[1]);
  }
}

template <typename T, bool kFast>
__global__ void __launch_bounds__(kEncThreads)
    k_encode(GeoDev g, SourceArgs src, long long n_rays, int S, int F, int grff_c,
             const float *grff_B, int ld, T *E, float *ray_l, const float *proj, float *ray_p) {
  extern __shared__ uint32_t enc_smem[];
  __shared__ Ray rays[kEncThreads];
  __shared__ float tfeat[kEncThreads][2 * kMaxFreq];
  __shared__ float sB[4 * kMaxGrff];
  for (int i = threadIdx.x; i < 4 * grff_c; i += blockDim.x) sB[i] = grff_B[i];
  const int words = ld * (int)sizeof(T) / 4;
  const int stride = words + 1;  // odd stride: conflict-free row writes
  const long long n = n_rays * S;
  const long long q0 = (long long)blockIdx.x * kEncThreads;
  const int tid = threadIdx.x;
  const bool ray_src = src.kind == kSrcTrainRays || src.kind == kSrcVirtualView;
  const long long r_first = q0 / S;
  long long q_last = q0 + kEncThreads - 1 < n - 1 ? q0 + kEncThreads - 1 : n - 1;
  const int nr_blk = (int)(q_last / S - r_first + 1);

  if (ray_src && tid < nr_blk) {
    long long r = r_first + tid;
    Ray ray = source_ray(g, src, r);
    rays[tid] = ray;
    if (grff_c == 0) coord_features<kFast>(ray.tbar, F, tfeat[tid]);
    if (r * S >= q0) {  // the block holding the ray's first sample reports it
      if (ray_l) ray_l[r] = (float)ray.l;
      if (ray_p) ray_p[r] = proj ? proj[src.idx[r]] : 0.0f;
    }
  }
  __syncthreads();

  const long long q = q0 + tid;
  uint32_t *row = enc_smem + tid * stride;
  if (q < n) {
    long long r = q / S;
    int j = (int)(q - r * S);
    double c[4];
    float sc[2 * kMaxFreq];
    if (ray_src) {
      int k = (int)(r - r_first);
      c[0] = rays[k].tbar;
      sample_coords(g, rays[k], j, S, c[1], c[2], c[3]);
      if (grff_c == 0)
        for (int l = 0; l < 2 * F; ++l) sc[l] = tfeat[k][l];
    } else {
      float len;
      source_coords(g, src, r, j, S, c, &len);
      if (ray_l) ray_l[r] = 1.0f;
      if (grff_c == 0) coord_features<kFast>(c[0], F, sc);
    }
    if (grff_c > 0) {
      grff_row<T, kFast>(row, c, sB, grff_c);
      for (int f = 2 * grff_c; f < ld; f += 2) FeatWriter<T>::put(row, f, 0.0f, 0.0f);
    } else {
    FeatWriter<T>::put(row, 0, (float)c[0], (float)c[1]);
    FeatWriter<T>::put(row, 2, (float)c[2], (float)c[3]);
    for (int l = 0; l < F; ++l) FeatWriter<T>::put(row, 4 + 2 * l, sc[2 * l], sc[2 * l + 1]);
    for (int k = 1; k < 4; ++k) {
      coord_features<kFast>(c[k], F, sc);
      for (int l = 0; l < F; ++l)
        FeatWriter<T>::put(row, 4 + 2 * F * k + 2 * l, sc[2 * l], sc[2 * l + 1]);
    }
    for (int f = 4 + 8 * F; f < ld; f += 2) FeatWriter<T>::put(row, f, 0.0f, 0.0f);
    }
  }
  __syncthreads();

  const long long rows = q_last - q0 + 1;
  uint32_t *dst = reinterpret_cast<uint32_t *>(E + q0 * ld);
  for (long long w = tid; w < rows * words; w += kEncThreads) {
    int rr = (int)(w / words), cc = (int)(w - (long long)rr * words);
    dst[w] = enc_smem[rr * stride + cc];
  }
}

template <typename T, bool kFast>
static void launch_encode(const GeoDev &g, const SourceArgs &src, long long n_rays, int S, int F,
                          int grff_c, const float *grff_B, int ld, T *E, float *ray_l,
                          const float *proj, float *ray_p, cudaStream_t st) {
  long long n = n_rays * S;
  int words = ld * (int)sizeof(T) / 4;
  size_t smem = (size_t)kEncThreads * (words + 1) * 4;
  static bool attr = false;
  if (!attr) {
    // rows of up to 256 FP32 features (GRFF with C = 128): 128 x 257 words
    cudaFuncSetAttribute(k_encode<T, kFast>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         160 * 1024);
    attr = true;
  }
  k_encode<T, kFast><<<ceil_div(n, kEncThreads), kEncThreads, smem, st>>>(
      g, src, n_rays, S, F, grff_c, grff_B, ld, E, ray_l, proj, ray_p);
}

void launch_encode_f32(const GeoDev &g, const SourceArgs &src, long long n_rays, int S,
                       int F, int grff_c, const float *grff_B, int ld, float *E, float *ray_l,
                       const float *proj, float *ray_p, cudaStream_t st) {
  launch_encode<float, false>(g, src, n_rays, S, F, grff_c, grff_B, ld, E, ray_l, proj, ray_p,
                              st);
}
void launch_encode_bf16(const GeoDev &g, const SourceArgs &src, long long n_rays, int S,
                        int F, int grff_c, const float *grff_B, int ld, __nv_bfloat16 *E,
                        float *ray_l, const float *proj, float *ray_p, cudaStream_t st) {
  launch_encode<__nv_bfloat16, true>(g, src, n_rays, S, F, grff_c, grff_B, ld, E, ray_l, proj,
                                     ray_p, st);
}

// ------------------------------------- output layer, forward model, loss
// One warp per ray; lanes split the W columns of each sample's dot product.
__global__ void k_out_segsum_f32(const float *zH, long long ld, int W, int act, int out_act,
                                 const float *w_out, const float *b_out, long long n_rays,
                                 int S, float mu0, const float *ray_l, const float *ray_p,
                                 float inv_B, int train, float *z_out, float *p_bar,
                                 float *sq, float *dz) {
  long long r = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (r >= n_rays) return;
  float bo = b_out[0];
  float sumM = 0.0f;
  for (int j = 0; j < S; ++j) {
    const float *row = zH + (r * S + j) * ld;
    float acc = 0.0f;
    for (int c = lane; c < W; c += 32) acc += act_f(row[c], act) * w_out[c];
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    float z = acc + bo;
    if (lane == 0) z_out[r * S + j] = z;
    sumM += out_f(z, out_act);
  }
  if (!p_bar) return;  // outputs only (ragged forward models sum them elsewhere)
  float l = ray_l[r];
  float pb = mu0 * (l / S) * sumM;
  if (lane == 0) {
    p_bar[r] = pb;
    if (train) {
      float res = pb - ray_p[r];
      sq[r] = res * res;
    }
  }
  if (!train) return;
  __syncwarp();
  float coef = 2.0f * inv_B * (pb - ray_p[r]) * mu0 * (l / S);
  for (int j = lane; j < S; j += 32) dz[r * S + j] = coef * out_grad_f(z_out[r * S + j], out_act);
}

void launch_out_segsum_f32(const float *zH, long long ld, int W, int act, int out_act,
                           const float *w_out, const float *b_out, long long n_rays, int S,
                           float mu0, const float *ray_l, const float *ray_p, float inv_B,
                           bool train, float *z_out, float *p_bar, float *sq, float *dz,
                           cudaStream_t st) {
  k_out_segsum_f32<<<ceil_div(n_rays * 32, 256), 256, 0, st>>>(
      zH, ld, W, act, out_act, w_out, b_out, n_rays, S, mu0, ray_l, ray_p, inv_B, train ? 1 : 0,
      z_out, p_bar, sq, dz);
}

// Warp-segmented forward model from per-sample outputs: each warp reduces
// one ray's S outputs in a fixed order (lane-strided partial sums, then a
// butterfly), then forms the residual and the per-sample adjoint.
__global__ void k_segsum(const float *z_out, int out_act, long long n_rays, int S, float mu0,
                         const float *ray_l, const float *ray_p, float inv_B, int train,
                         float *p_bar, float *sq, float *dz) {
  long long r = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (r >= n_rays) return;
  const float *z = z_out + r * S;
  float s = 0.0f;
  for (int j = lane; j < S; j += 32) s += out_f(z[j], out_act);
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  float l = ray_l[r];
  float pb = mu0 * (l / S) * s;
  if (lane == 0) {
    p_bar[r] = pb;
    if (train) {
      float res = pb - ray_p[r];
      sq[r] = res * res;
    }
  }
  if (!train) return;
  float coef = 2.0f * inv_B * (pb - ray_p[r]) * mu0 * (l / S);
  for (int j = lane; j < S; j += 32) dz[r * S + j] = coef * out_grad_f(z[j], out_act);
}

void launch_segsum(const float *z_out, int out_act, long long n_rays, int S, float mu0,
                   const float *ray_l, const float *ray_p, float inv_B, bool train,
                   float *p_bar, float *sq, float *dz, cudaStream_t st) {
  k_segsum<<<ceil_div(n_rays * 32, 256), 256, 0, st>>>(z_out, out_act, n_rays, S, mu0, ray_l,
                                                       ray_p, inv_B, train ? 1 : 0, p_bar, sq,
                                                       dz);
}

__global__ void k_out_delta_f32(const float *dz, const float *w_out, const float *zH,
                                long long ld, int W, int act, long long n, float *D) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= n * W) return;
  long long s = q / W;
  int c = (int)(q - s * W);
  D[s * W + c] = dz[s] * w_out[c] * act_grad_f(zH[s * ld + c], act);
}
void launch_out_delta_f32(const float *dz, const float *w_out, const float *zH, long long ld,
                          int W, int act, long long n, float *D, cudaStream_t st) {
  k_out_delta_f32<<<ceil_div(n * W, 256), 256, 0, st>>>(dz, w_out, zH, ld, W, act, n, D);
}

// ------------------------------------------------------ column sums
int colsum_splits(long long rows) {
  long long s = (rows + 2047) / 2048;
  return (int)(s < 1 ? 1 : (s > 1184 ? 1184 : s));
}

__global__ void k_colsum(const float *X, long long ld, int C, long long rows, const float *w,
                         int apply_act, int act, int splits, float *part) {
  int z = blockIdx.y;
  long long per = (rows + splits - 1) / splits;
  long long r0 = z * per, r1 = r0 + per < rows ? r0 + per : rows;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
    float acc = 0.0f, blk = 0.0f;     // blocked summation, blocks of 256 rows
    for (long long r = r0; r < r1; ++r) {
      float x = X[r * ld + c];
      if (apply_act) x = act_f(x, act);
      blk += w ? w[r] * x : x;
      if (((r - r0) & 255) == 255) {
        acc += blk;
        blk = 0.0f;
      }
    }
    part[(long long)z * C + c] = acc + blk;
  }
}
// One column (e.g. the output bias gradient sum of dz): all 256 threads of a
// block share the rows of its split (strided), then a fixed shared-memory
// tree adds the thread sums.
__global__ void __launch_bounds__(256)
    k_colsum1(const float *X, long long ld, long long rows, const float *w, int apply_act,
              int act, int splits, float *part) {
  __shared__ float red[256];
  const int z = blockIdx.x;
  const long long per = (rows + splits - 1) / splits;
  const long long r0 = z * per, r1 = r0 + per < rows ? r0 + per : rows;
  float acc = 0.0f;
  for (long long r = r0 + threadIdx.x; r < r1; r += 256) {
    float x = X[r * ld];
    if (apply_act) x = act_f(x, act);
    acc += w ? w[r] * x : x;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[z] = red[0];
}

void launch_colsum(const float *X, long long ld, int C, long long rows, const float *w,
                   bool apply_act, int act, int splits, float *part, cudaStream_t st) {
  if (C == 1) {
    k_colsum1<<<splits, 256, 0, st>>>(X, ld, rows, w, apply_act ? 1 : 0, act, splits, part);
    return;
  }
  dim3 grid(ceil_div(C, 256), splits);
  k_colsum<<<grid, 256, 0, st>>>(X, ld, C, rows, w, apply_act ? 1 : 0, act, splits, part);
}

// out[c] (+)= sum over z of part[z][c] in a fixed order: a block takes 32
// consecutive elements; each of its 8 warps sums the splits z = g, g + 8, ...
// of them (coalesced 128-byte rows, 8 times the loads in flight of one
// thread per element), and one thread per element adds the 8 warp sums in
// order.
__global__ void __launch_bounds__(256)
    k_reduce_partials(const float *part, int splits, long long C, float *out, int accumulate) {
  __shared__ float red[8][33];
  const int e = threadIdx.x & 31, g = threadIdx.x >> 5;
  const long long c = blockIdx.x * 32LL + e;
  float s = 0.0f;
  if (c < C)
    for (int z = g; z < splits; z += 8) s += part[(long long)z * C + c];
  red[g][e] = s;
  __syncthreads();
  if (g == 0 && c < C) {
    float t = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += red[k][e];
    out[c] = (accumulate ? out[c] : 0.0f) + t;
  }
}
void launch_reduce_partials(const float *part, int splits, long long C, float *out,
                            bool accumulate, cudaStream_t st) {
  k_reduce_partials<<<ceil_div(C, 32), 256, 0, st>>>(part, splits, C, out, accumulate ? 1 : 0);
}

// One block, fixed order: strided partial sums then a tree.
__global__ void k_loss_sum(const float *sq, long long n, float inv_B, float *loss,
                           int accumulate) {
  __shared__ float red[1024];
  float s = 0.0f;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) s += sq[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss[0] = (accumulate ? loss[0] : 0.0f) + inv_B * red[0];
}
void launch_loss_sum(const float *sq, long long n, float inv_B, float *loss, bool accumulate,
                     cudaStream_t st) {
  k_loss_sum<<<1, 1024, 0, st>>>(sq, n, inv_B, loss, accumulate ? 1 : 0);
}

// ------------------------------------------------------------------- Adam
__global__ void k_adam(float *theta, float *m, float *v, const float *g, long long P, float lr,
                       float beta1, float beta2, float eps, float bc1, float bc2) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= P) return;
  float gi = g[i];
  float mi = beta1 * m[i] + (1.0f - beta1) * gi;
  float vi = beta2 * v[i] + (1.0f - beta2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  theta[i] -= lr * (mi * bc1) / (sqrtf(vi * bc2) + eps);
}
void launch_adam(float *theta, float *m, float *v, const float *g, long long P, float lr,
                 float beta1, float beta2, float eps, float bc1, float bc2, cudaStream_t st) {
  k_adam<<<ceil_div(P, 256), 256, 0, st>>>(theta, m, v, g, P, lr, beta1, beta2, eps, bc1, bc2);
}


// Adam of a graph-replayed step: the same update as k_adam with the step's
// learning rate and bias corrections read from a host-filled table, entry
// (*step - *step0).
__global__ void k_adam_tab(float *theta, float *m, float *v, const float *g, long long P,
                           float beta1, float beta2, float eps, const float *tab,
                           const long long *step, const long long *step0) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= P) return;
  const long long k = *step - *step0;
  const float lr = tab[3 * k], bc1 = tab[3 * k + 1], bc2 = tab[3 * k + 2];
  float gi = g[i];
  float mi = beta1 * m[i] + (1.0f - beta1) * gi;
  float vi = beta2 * v[i] + (1.0f - beta2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  theta[i] -= lr * (mi * bc1) / (sqrtf(vi * bc2) + eps);
}
void launch_adam_tab(float *theta, float *m, float *v, const float *g, long long P, float beta1,
                     float beta2, float eps, const float *tab, const long long *step,
                     const long long *step0, cudaStream_t st) {
  k_adam_tab<<<ceil_div(P, 256), 256, 0, st>>>(theta, m, v, g, P, beta1, beta2, eps, tab, step,
                                               step0);
}

// *step += 1 (the end of a graph-replayed step).
__global__ void k_step_inc(long long *step) {
  if (threadIdx.x == 0) *step += 1;
}
void launch_step_inc(long long *step, cudaStream_t st) { k_step_inc<<<1, 32, 0, st>>>(step); }

// out[i] = g[i] * (*scale): the gradient of (scale x L) from that of L (the
// upstream factor an autograd backward passes in).
__global__ void k_scale_by(const float *g, long long P, const float *scale, float *out) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < P) out[i] = g[i] * scale[0];
}
void launch_scale_by(const float *g, long long P, const float *scale, float *out,
                     cudaStream_t st) {
  k_scale_by<<<ceil_div(P, 256), 256, 0, st>>>(g, P, scale, out);
}

}  // namespace dinr
