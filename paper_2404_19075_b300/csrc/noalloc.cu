// dinr_phantom_project_noalloc: the phantom projector for callers that
// cannot allocate device memory (see include/dinr.h).
//
// The per-view table and the ellipsoid parameters that dinr_phantom_project
// stages in freshly allocated device memory live here in one file-scope
// device array instead. Host code must not pass the array's name to a
// kernel (on the host it is only a stand-in symbol); its device address is
// looked up once per device with cudaGetSymbolAddress and cached.
#include "context.cuh"

#include <cmath>
#include <mutex>

using namespace dinr;

namespace {

constexpr int kMaxViews = 4096;
constexpr int kMaxEll = 1024;
constexpr int kMaxDevices = 64;

// Layout of the scratch array, in doubles.
constexpr int kOffAngle = 0;                          // [kMaxViews] raw angles
constexpr int kOffTime = kOffAngle + kMaxViews;       // [kMaxViews] raw times
constexpr int kOffCs = kOffTime + kMaxViews;          // [kMaxViews] (cos, sin)
constexpr int kOffTbar = kOffCs + 2 * kMaxViews;      // [kMaxViews] normalised times
constexpr int kOffCentre = kOffTbar + kMaxViews;      // [3 kMaxEll]
constexpr int kOffAxes = kOffCentre + 3 * kMaxEll;    // [3 kMaxEll]
constexpr int kOffRho = kOffAxes + 3 * kMaxEll;       // [kMaxEll]
constexpr int kOffVel = kOffRho + kMaxEll;            // [3 kMaxEll]
constexpr int kOffEll = kOffVel + 3 * kMaxEll;        // [10 kMaxEll] packed ellipsoids
constexpr int kScratchDoubles = kOffEll + 10 * kMaxEll;  // 40,960 doubles = 320 KiB

static __device__ __align__(256) double g_phantom_scratch[kScratchDoubles];

std::mutex g_mu;
double *g_dev_ptr[kMaxDevices] = {};

// Per-view (cos, sin, normalised time) in FP64 and the packed ellipsoid
// records (centre, axes, rho, velocity) that k_phantom reads.
__global__ void k_prep(int n_views, double t0, double t1, int n_ell, int has_vel, double *s) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_views) {
    double a = s[kOffAngle + i];
    s[kOffCs + 2 * i] = cos(a);
    s[kOffCs + 2 * i + 1] = sin(a);
    s[kOffTbar + i] = 2.0 * (s[kOffTime + i] - t0) / (t1 - t0) - 1.0;
  }
  if (i < n_ell) {
    double *e = s + kOffEll + 10 * i;
    for (int d = 0; d < 3; ++d) {
      e[d] = s[kOffCentre + 3 * i + d];
      e[3 + d] = s[kOffAxes + 3 * i + d];
      e[7 + d] = has_vel ? s[kOffVel + 3 * i + d] : 0.0;
    }
    e[6] = s[kOffRho + i];
  }
}

}  // namespace

dinr_status dinr_phantom_project_noalloc(const dinr_geometry *geom, int n_ell,
                                         const double *centre, const double *axes,
                                         const double *rho, const double *vel, double growth,
                                         const int64_t *idx, int64_t n, float *out,
                                         void *cuda_stream) {
  const dinr_geometry *g = geom;
  if (!g || !g->view_angle || !g->view_time || n < 0 || !out || n_ell < 0 ||
      (n_ell > 0 && (!centre || !axes || !rho)) ||
      (g->beam != DINR_BEAM_PARALLEL && g->beam != DINR_BEAM_CONE) || g->n_views < 1 ||
      g->det_rows < 1 || g->det_cols < 1 || !(g->det_pitch_u > 0) || !(g->det_pitch_v > 0) ||
      !(g->fov_r > 0) || !(g->fov_z1 > g->fov_z0) || !(g->t1 > g->t0) ||
      (g->beam == DINR_BEAM_CONE && (!(g->sod > g->fov_r) || !(g->sdd > g->sod))))
    return (dinr_status)dinr_fail(nullptr, DINR_ERR_ARG, "invalid phantom request");
  if (g->n_views > kMaxViews || n_ell > kMaxEll)
    return (dinr_status)dinr_fail(nullptr, DINR_ERR_ARG,
                                  "dinr_phantom_project_noalloc supports at most %d views and "
                                  "%d ellipsoids (got %d and %d)",
                                  kMaxViews, kMaxEll, g->n_views, n_ell);
  if (n == 0) return DINR_OK;

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return (dinr_status)dinr_fail(nullptr, DINR_ERR_CUDA, "no usable current device");
  double *s = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev_ptr[dev]) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_phantom_scratch);
      if (e != cudaSuccess)
        return (dinr_status)dinr_fail(nullptr, DINR_ERR_CUDA, "cudaGetSymbolAddress: %s",
                                      cudaGetErrorString(e));
      g_dev_ptr[dev] = static_cast<double *>(p);
    }
    s = g_dev_ptr[dev];
  }

  cudaStream_t st = (cudaStream_t)cuda_stream;
  const size_t d8 = sizeof(double);
  const int M = g->n_views;
  struct Copy {
    int off;
    const double *src;
    size_t count;
  } copies[] = {{kOffAngle, g->view_angle, (size_t)M},
                {kOffTime, g->view_time, (size_t)M},
                {kOffCentre, centre, 3 * (size_t)n_ell},
                {kOffAxes, axes, 3 * (size_t)n_ell},
                {kOffRho, rho, (size_t)n_ell},
                {kOffVel, vel, 3 * (size_t)n_ell}};
  for (const Copy &c : copies) {
    if (!c.src || c.count == 0) continue;
    e = cudaMemcpyAsync(s + c.off, c.src, c.count * d8, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess)
      return (dinr_status)dinr_fail(nullptr, DINR_ERR_CUDA, "staging copy: %s",
                                    cudaGetErrorString(e));
  }
  int m = M > n_ell ? M : n_ell;
  k_prep<<<(m + 127) / 128, 128, 0, st>>>(M, g->t0, g->t1, n_ell, vel ? 1 : 0, s);

  GeoDev d{};
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
  d.mu0 = (float)g->mu0;
  d.view_cs = reinterpret_cast<const double2 *>(s + kOffCs);
  d.view_tbar = s + kOffTbar;
  launch_phantom(d, s + kOffTime, n_ell, s + kOffEll, growth, (const long long *)idx, n, out, st);
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return (dinr_status)dinr_fail(nullptr, DINR_ERR_CUDA, "phantom launch: %s",
                                  cudaGetErrorString(e));
  return DINR_OK;
}
