// dinr_phantom_project_noalloc: the phantom projector for callers that
// cannot allocate device memory (see include/dinr.h).
//
// The per-view table and the ellipsoid records that dinr_phantom_project
// stages in freshly allocated device memory live here in one file-scope
// device array instead. Host code must not pass the array's name to a
// kernel (on the host it is only a stand-in symbol); its device address is
// looked up with cudaGetSymbolAddress, with the device current, once per
// device context, and cached.
//
// The table is built on the host (the same FP64 cos, sin and time
// normalisation as dinr_phantom_project) in a static host buffer, under a
// mutex, and copied with one cudaMemcpyAsync per part. The buffer is
// ordinary pageable memory, so each copy has taken its bytes out of it when
// cudaMemcpyAsync returns; the caller's arrays are read only during the call.
#include "context.cuh"

#include <cmath>
#include <cstring>
#include <mutex>

using namespace dinr;

namespace {

constexpr int kMaxViews = 4096;
constexpr int kMaxEll = 1024;
constexpr int kMaxDevices = 64;

// Layout of the scratch array, in doubles.
constexpr int kOffCs = 0;                              // [kMaxViews] (cos, sin) of each view
constexpr int kOffTbar = kOffCs + 2 * kMaxViews;       // [kMaxViews] normalised view times
constexpr int kOffTime = kOffTbar + kMaxViews;         // [kMaxViews] view times
constexpr int kOffEll = kOffTime + kMaxViews;          // [10 kMaxEll] packed ellipsoids
constexpr int kScratchDoubles = kOffEll + 10 * kMaxEll;  // 26,624 doubles = 208 KiB

static __device__ __align__(256) double g_phantom_scratch[kScratchDoubles];

// Host image of the scratch array (pageable), filled under g_mu.
double g_host_image[kScratchDoubles];

std::mutex g_mu;
struct DevSlot {
  unsigned long long ctx_id = 0;  // context the address belongs to (0: none yet)
  double *ptr = nullptr;
};
DevSlot g_slot[kMaxDevices];

typedef int (*PfnCtxGetCurrent)(void **ctx);
typedef int (*PfnCtxGetId)(void *ctx, unsigned long long *id);

// Unique id of the calling thread's current context (0 if there is none or
// the driver cannot say). A device reset or a new context gets a new id.
unsigned long long current_ctx_id() {
  static PfnCtxGetCurrent get_current = nullptr;
  static PfnCtxGetId get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<PfnCtxGetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<PfnCtxGetId>(f);
    looked_up = true;
  }
  if (!get_current || !get_id) return 0;
  void *ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

}  // namespace

dinr_status dinr_phantom_project_noalloc(const dinr_geometry *geom, int n_ell,
                                         const double *centre, const double *axes,
                                         const double *rho, const double *vel, double growth,
                                         const int64_t *idx, int64_t n, float *out,
                                         void *cuda_stream) {
  const dinr_geometry *g = geom;
  if (!dinr_geometry_valid(g) || n < 0 || !out || n_ell < 0 ||
      (n_ell > 0 && (!centre || !axes || !rho)))
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
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int M = g->n_views;
  double *s = nullptr;
  std::lock_guard<std::mutex> lock(g_mu);
  {
    // The address is looked up again when the current context is not the
    // one it was taken in (a device reset gives the device a new context).
    const unsigned long long id = current_ctx_id();
    DevSlot &slot = g_slot[dev];
    if (!slot.ptr || id == 0 || slot.ctx_id != id) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_phantom_scratch);
      if (e != cudaSuccess)
        return (dinr_status)dinr_fail(nullptr, DINR_ERR_CUDA, "cudaGetSymbolAddress: %s",
                                      cudaGetErrorString(e));
      slot.ptr = static_cast<double *>(p);
      slot.ctx_id = current_ctx_id();
    }
    s = slot.ptr;
  }

  // Host image: per view (cos, sin), normalised time and time in FP64 (as
  // dinr_phantom_project forms them), then the packed ellipsoid records
  // (centre, semi-axes, rho, velocity) that the phantom kernel reads.
  double *h = g_host_image;
  for (int m = 0; m < M; ++m) {
    h[kOffCs + 2 * m] = std::cos(g->view_angle[m]);
    h[kOffCs + 2 * m + 1] = std::sin(g->view_angle[m]);
    h[kOffTbar + m] = 2.0 * (g->view_time[m] - g->t0) / (g->t1 - g->t0) - 1.0;
    h[kOffTime + m] = g->view_time[m];
  }
  for (int k = 0; k < n_ell; ++k) {
    double *r = h + kOffEll + 10 * k;
    for (int d = 0; d < 3; ++d) {
      r[d] = centre[3 * k + d];
      r[3 + d] = axes[3 * k + d];
      r[7 + d] = vel ? vel[3 * k + d] : 0.0;
    }
    r[6] = rho[k];
  }
  struct Part {
    int off;
    size_t count;
  } parts[] = {{kOffCs, 2 * (size_t)M}, {kOffTbar, (size_t)M}, {kOffTime, (size_t)M},
               {kOffEll, 10 * (size_t)n_ell}};
  for (const Part &q : parts) {
    if (q.count == 0) continue;
    e = cudaMemcpyAsync(s + q.off, h + q.off, q.count * sizeof(double), cudaMemcpyHostToDevice,
                        st);
    if (e != cudaSuccess)
      return (dinr_status)dinr_fail(nullptr, DINR_ERR_CUDA, "staging copy: %s",
                                    cudaGetErrorString(e));
  }

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
