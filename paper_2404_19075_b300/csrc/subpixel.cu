// App. A forward model (see subpixel.cuh).
//
// A pass of n_pix pixels has K = n_pix D^2 sub-rays. One thread per sub-ray
// sets it up in FP64 (decode, sub-pixel centre, rotation, FOV chord, sample
// count ceil(l / spacing), normalised first sample and step); an exclusive
// scan of the counts gives each ray's first sample (a pixel's rays, and so
// its samples, are contiguous); one warp per ray writes the owner index of
// its samples. Encoders take sample q's coordinates from its owner's record;
// the forward model sums a pixel's samples with one warp per pixel.
#include "subpixel.cuh"

#include <cmath>

using namespace dinr;

namespace {

constexpr int kScan = 1024;  // elements per scan block

struct SubpixWs {
  long long k_cap = 0, s_cap = 0;
  double *rec64 = nullptr;      // [K][8] tbar, first sample (z, y, x), step (z, y, x), l
  float *rec32 = nullptr;       // [K][8] the same in FP32 (chain encoders)
  int *cnt = nullptr;           // [K] samples per ray
  long long *first = nullptr;   // [K + 1] first sample of each ray; first[K] = total
  long long *bsum = nullptr;    // [K / kScan + 2] scan block sums
  float *wl = nullptr;          // [K] mu0 * l of each ray (FP32 weight)
  float *pix_p = nullptr;       // [n_pix] measured p of each pixel
  int *owner = nullptr;         // [samples] ray of each sample
  long long *host_total = nullptr;  // pinned
  int n_pix = 0;
};

SubpixWs *W_(dinr_ctx *c) { return static_cast<SubpixWs *>(c->subpix); }

__global__ void k_subrays(GeoDev g, const long long *idx, int n_pix, const float *proj,
                          double *rec64, float *rec32, int *cnt, float *wl, float *pix_p) {
  const int D = g.D, D2 = D * D;
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= (long long)n_pix * D2) return;
  const int p = (int)(k / D2), sub = (int)(k - (long long)p * D2);
  const int a = sub / D, b = sub - a * D;  // (row, column) sub-pixel
  const long long i = idx[p];
  const long long m = i / g.n_pixels, n = i - m * g.n_pixels;
  const int row = (int)(n / g.det_cols), col = (int)(n - (long long)row * g.det_cols);
  const double u = g.ou + (col + (b + 0.5) / D) * g.pu;
  const double v = g.ov + (row + (a + 0.5) / D) * g.pv;
  const double2 cs = g.view_cs[m];
  const Ray r = ray_at(g, u, v, cs.x, cs.y, g.view_tbar[m]);
  int cn = 0;
  if (r.l > 0.0) {
    cn = (int)ceil(r.l / g.spacing);
    if (cn < 1) cn = 1;
  }
  cnt[k] = cn;
  wl[k] = g.mu0 * (float)r.l;
  const double step = cn > 0 ? r.l / cn : 0.0;
  const double s = r.s0 + 0.5 * step;
  const double R[8] = {r.tbar,
                       (r.oz + s * r.dz) * g.zs + g.zb,
                       (r.oy + s * r.dy) * g.inv_R,
                       (r.ox + s * r.dx) * g.inv_R,
                       step * r.dz * g.zs,
                       step * r.dy * g.inv_R,
                       step * r.dx * g.inv_R,
                       r.l};
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    rec64[8 * k + e] = R[e];
    rec32[8 * k + e] = (float)R[e];
  }
  if (sub == 0) pix_p[p] = proj ? proj[i] : 0.0f;
}

// Exclusive scan of cnt[0..K) into first[], kScan elements per block;
// bsum[b] = the block's total.
__global__ void __launch_bounds__(kScan) k_scan_block(const int *cnt, long long K,
                                                      long long *first, long long *bsum) {
  __shared__ long long sh[kScan];
  const long long q = blockIdx.x * (long long)kScan + threadIdx.x;
  const long long x = q < K ? cnt[q] : 0;
  sh[threadIdx.x] = x;
  __syncthreads();
  for (int off = 1; off < kScan; off <<= 1) {  // inclusive Hillis-Steele
    long long y = threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
    __syncthreads();
    sh[threadIdx.x] += y;
    __syncthreads();
  }
  if (q < K) first[q] = sh[threadIdx.x] - x;
  if (threadIdx.x == kScan - 1) bsum[blockIdx.x] = sh[kScan - 1];
}

// Exclusive scan of the block totals (one block; nb <= kScan); the total
// goes to first[K] and bsum[nb].
__global__ void __launch_bounds__(kScan) k_scan_sums(long long *bsum, int nb, long long *first,
                                                     long long K) {
  __shared__ long long sh[kScan];
  const long long x = threadIdx.x < nb ? bsum[threadIdx.x] : 0;
  sh[threadIdx.x] = x;
  __syncthreads();
  for (int off = 1; off < kScan; off <<= 1) {
    long long y = threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
    __syncthreads();
    sh[threadIdx.x] += y;
    __syncthreads();
  }
  if (threadIdx.x < nb) bsum[threadIdx.x] = sh[threadIdx.x] - x;
  if (threadIdx.x == kScan - 1) {
    first[K] = sh[kScan - 1];
    bsum[nb] = sh[kScan - 1];
  }
}

__global__ void k_scan_add(long long *first, const long long *bsum, long long K) {
  const long long q = blockIdx.x * (long long)kScan + threadIdx.x;
  if (q < K) first[q] += bsum[blockIdx.x];
}

// One warp per ray: owner[s] = k for the ray's samples.
__global__ void k_owner(const long long *first, long long K, int *owner) {
  const long long k = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  if (k >= K) return;
  const long long f = first[k], n = first[k + 1] - f;
  for (long long j = lane; j < n; j += 32) owner[f + j] = (int)k;
}

// One warp per pixel: p_bar = (1/|Phi|) sum over the pixel's samples of
// mu0 l(ray) out(z), summed in a fixed order (lane-strided per ray, then a
// shuffle tree), 0 for a pixel without samples; with train, the loss term
// and dL/dz of every sample.
__global__ void k_segsum_subpix(const float *z_out, int out_act, int n_pix, int D2,
                                const long long *first, const float *wl, const float *pix_p,
                                float inv_B, int train, float *p_bar, float *sq, float *dz) {
  const long long p = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  if (p >= n_pix) return;
  const long long k0 = p * D2;
  float acc = 0.0f;
  for (int r = 0; r < D2; ++r) {
    const long long f = first[k0 + r], n = first[k0 + r + 1] - f;
    const float w = wl[k0 + r];
    float part = 0.0f;
    for (long long j = lane; j < n; j += 32) part += out_f(z_out[f + j], out_act);
    acc = fmaf(w, part, acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  const long long N = first[k0 + D2] - first[k0];
  const float pb = N > 0 ? acc / (float)N : 0.0f;
  const float res = pb - pix_p[p];
  if (lane == 0) {
    p_bar[p] = pb;
    if (sq) sq[p] = res * res;
  }
  if (train && N > 0) {
    const float cf = 2.0f * inv_B * res / (float)N;
    for (int r = 0; r < D2; ++r) {
      const long long f = first[k0 + r], n = first[k0 + r + 1] - f;
      const float w = cf * wl[k0 + r];
      for (long long j = lane; j < n; j += 32) dz[f + j] = w * out_grad_f(z_out[f + j], out_act);
    }
  }
}

}  // namespace

dinr_status subpix_alloc(dinr_ctx *c) {
  if (c->geo.D <= 0) return DINR_OK;
  SubpixWs *w = new SubpixWs();
  c->subpix = w;
  const long long K = (long long)c->chunk_rays * c->geo.D * c->geo.D;
  const long long S = (long long)c->chunk_rays * c->S;
  if ((K + kScan - 1) / kScan > kScan)
    return (dinr_status)dinr_fail(c, DINR_ERR_UNSUPPORTED, "too many sub-rays per pass");
  w->k_cap = K;
  w->s_cap = S;
  bool ok = true;
  auto grab = [&](void **p, size_t bytes) {
    if (!ok) return;
    if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) {
      cudaGetLastError();
      ok = false;
      return;
    }
    c->allocs.push_back(*p);
  };
  grab((void **)&w->rec64, sizeof(double) * 8 * K);
  grab((void **)&w->rec32, sizeof(float) * 8 * K);
  grab((void **)&w->cnt, sizeof(int) * K);
  grab((void **)&w->first, sizeof(long long) * (K + 1));
  grab((void **)&w->bsum, sizeof(long long) * (K / kScan + 2));
  grab((void **)&w->wl, sizeof(float) * K);
  grab((void **)&w->pix_p, sizeof(float) * c->chunk_rays);
  grab((void **)&w->owner, sizeof(int) * S);
  if (ok && cudaMallocHost((void **)&w->host_total, sizeof(long long)) != cudaSuccess) {
    cudaGetLastError();
    ok = false;
  }
  if (!ok) return (dinr_status)dinr_fail(c, DINR_ERR_OOM, "sub-ray workspace allocation failed");
  return DINR_OK;
}

void subpix_free(dinr_ctx *c) {
  SubpixWs *w = W_(c);
  if (!w) return;
  if (w->host_total) cudaFreeHost(w->host_total);
  delete w;
  c->subpix = nullptr;
}

dinr_status subpix_setup(dinr_ctx *c, const long long *idx, int n_pix, const float *proj,
                         long long *n_samples) {
  SubpixWs *w = W_(c);
  const long long K = (long long)n_pix * c->geo.D * c->geo.D;
  if (!w || K > w->k_cap)
    return (dinr_status)dinr_fail(c, DINR_ERR_STATE, "sub-ray workspace too small");
  k_subrays<<<(int)ceil_div(K, 128), 128, 0, c->st>>>(c->geo, idx, n_pix, proj, w->rec64,
                                                        w->rec32, w->cnt, w->wl, w->pix_p);
  const int nb = (int)ceil_div(K, kScan);
  k_scan_block<<<nb, kScan, 0, c->st>>>(w->cnt, K, w->first, w->bsum);
  k_scan_sums<<<1, kScan, 0, c->st>>>(w->bsum, nb, w->first, K);
  k_scan_add<<<nb, kScan, 0, c->st>>>(w->first, w->bsum, K);
  c->launches += 4;
  cudaError_t e = cudaMemcpyAsync(w->host_total, w->first + K, sizeof(long long),
                                  cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess)
    return (dinr_status)dinr_fail(c, DINR_ERR_CUDA, "sub-ray setup: %s", cudaGetErrorString(e));
  const long long total = *w->host_total;
  if (total > w->s_cap)
    return (dinr_status)dinr_fail(c, DINR_ERR_STATE, "sub-ray samples exceed the workspace");
  k_owner<<<(int)ceil_div(K * 32, 256), 256, 0, c->st>>>(w->first, K, w->owner);
  ++c->launches;
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return (dinr_status)dinr_fail(c, DINR_ERR_CUDA, "sub-ray setup: %s", cudaGetErrorString(e));
  w->n_pix = n_pix;
  *n_samples = total;
  return DINR_OK;
}

SourceArgs subpix_source(dinr_ctx *c) {
  SubpixWs *w = W_(c);
  SourceArgs s{};
  s.kind = kSrcSubRays;
  s.owner = w->owner;
  s.sfirst = w->first;
  s.srec = w->rec64;
  s.srec32 = w->rec32;
  return s;
}

dinr_status subpix_segsum(dinr_ctx *c, const float *z_out, int n_pix, float inv_B, bool train,
                          float *p_bar, float *sq, float *dz) {
  SubpixWs *w = W_(c);
  const int D2 = c->geo.D * c->geo.D;
  k_segsum_subpix<<<(int)ceil_div((long long)n_pix * 32, 256), 256, 0, c->st>>>(
      z_out, c->out_act, n_pix, D2, w->first, w->wl, w->pix_p, inv_B, train ? 1 : 0, p_bar, sq,
      dz);
  ++c->launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return (dinr_status)dinr_fail(c, DINR_ERR_CUDA, "sub-ray segment sums: %s",
                                  cudaGetErrorString(e));
  return DINR_OK;
}
