// Shared device-side definitions of libdinr: geometry of a ray (Sec. III,
// App. A), coordinate normalisation and Fourier features (App. B), the
// SplitMix64 mixer, activations.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace dinr {

constexpr int kMaxFreq = 16;
constexpr int kMaxGrff = 128;  // GRFF frequencies C (2C = 256 features)

// Geometry as the kernels see it. Per-view angle cosines/sines and
// normalised times are computed on the host in FP64 at creation.
struct GeoDev {
  int beam;                 // 0 parallel, 1 cone
  int n_views, det_rows, det_cols;
  long long n_pixels, n_proj;
  double pu, pv, ou, ov;    // detector pitch and offset
  double sod, sdd;
  double R, z0, z1;         // FOV cylinder
  double inv_R, zs, zb;     // x_bar = x * inv_R, z_bar = z * zs + zb
  int S;                    // samples per ray
  int D;                    // App. A sub-pixel rays per pixel side (0: one ray, S samples)
  double spacing;           // App. A sample spacing: back-projected pixel / D
  float mu0;
  const double2 *view_cs;   // (cos theta_m, sin theta_m)
  const double *view_tbar;  // 2 (T_m - t0) / (t1 - t0) - 1
};

struct Ray {
  double ox, oy, oz, dx, dy, dz;  // origin and unit direction
  double s0, l;                   // FOV chord start and length
  double tbar;                    // normalised time of the view
};

// Chord of o + s d through the FOV cylinder and z-slab (Sec. III: only the
// region inside the cylindrical FOV contributes). Empty chords give s0 = 0,
// l = 0.
__device__ __forceinline__ void fov_chord(const GeoDev &g, Ray &r) {
  double a = r.dx * r.dx + r.dy * r.dy;
  double b = 2.0 * (r.ox * r.dx + r.oy * r.dy);
  double c = r.ox * r.ox + r.oy * r.oy - g.R * g.R;
  double disc = b * b - 4.0 * a * c;
  r.s0 = 0.0;
  r.l = 0.0;
  if (!(disc > 0.0) || !(a > 0.0)) return;
  double sq = sqrt(disc);
  double lo = (-b - sq) / (2.0 * a);
  double hi = (-b + sq) / (2.0 * a);
  if (r.dz != 0.0) {
    double za = (g.z0 - r.oz) / r.dz, zb = (g.z1 - r.oz) / r.dz;
    lo = fmax(lo, fmin(za, zb));
    hi = fmin(hi, fmax(za, zb));
  } else if (r.oz < g.z0 || r.oz > g.z1) {
    return;
  }
  if (hi > lo) {
    r.s0 = lo;
    r.l = hi - lo;
  }
}

// Ray of a detector point (u, v) of a view with rotation (c, s): the
// source/detector pair is rotated by -theta (Sec. III).
__device__ __forceinline__ Ray ray_at(const GeoDev &g, double u, double v,
                                      double c, double s, double tbar) {
  double ax, ay, az, bx, by, bz;  // local origin (a) and direction (b)
  if (g.beam == 0) {
    ax = u; ay = 0.0; az = v;
    bx = 0.0; by = 1.0; bz = 0.0;
  } else {
    ax = 0.0; ay = -g.sod; az = 0.0;
    double n = 1.0 / sqrt(u * u + g.sdd * g.sdd + v * v);
    bx = u * n; by = g.sdd * n; bz = v * n;
  }
  Ray r;
  r.ox = ax * c + ay * s;  r.oy = -ax * s + ay * c;  r.oz = az;
  r.dx = bx * c + by * s;  r.dy = -bx * s + by * c;  r.dz = bz;
  r.tbar = tbar;
  fov_chord(g, r);
  return r;
}

// Sec. III decode: m = i div N, n = i mod N, (row, col) = (n div cols, n mod cols).
__device__ __forceinline__ Ray make_ray(const GeoDev &g, long long i) {
  long long m = i / g.n_pixels;
  long long n = i - m * g.n_pixels;
  int row = (int)(n / g.det_cols);
  int col = (int)(n - (long long)row * g.det_cols);
  double u = g.ou + (col + 0.5) * g.pu;
  double v = g.ov + (row + 0.5) * g.pv;
  double2 cs = g.view_cs[m];
  return ray_at(g, u, v, cs.x, cs.y, g.view_tbar[m]);
}

// Normalised sample j of S on a ray (App. A midpoints; App. B item 1), FP64.
__device__ __forceinline__ void sample_coords(const GeoDev &g, const Ray &r, int j, int S,
                                              double &zb, double &yb, double &xb) {
  double s = r.s0 + (j + 0.5) * (r.l / S);
  double x = r.ox + s * r.dx, y = r.oy + s * r.dy, z = r.oz + s * r.dz;
  xb = x * g.inv_R;
  yb = y * g.inv_R;
  zb = z * g.zs + g.zb;
}

// sin(2^l pi c) and cos(2^l pi c) for one coordinate. c is split into
// FP32 hi + lo parts; 2^l * hi is exact, and subtracting the nearest even
// integer from it is exact, so the phase handed to sincospif carries only
// the rounding of the final add (about 1e-7 of a half-turn) at every octave.
__device__ __forceinline__ void octave_features(double c, int F, float *sc) {
  float hi = (float)c;
  float lo = (float)(c - (double)hi);
  float scale = 1.0f;
  for (int l = 0; l < F; ++l) {
    float a = hi * scale;
    float n = 2.0f * rintf(0.5f * a);
    float y = (a - n) + lo * scale;
    float sv, cv;
    sincospif(y, &sv, &cv);
    sc[2 * l] = sv;
    sc[2 * l + 1] = cv;
    scale *= 2.0f;
  }
}

// SplitMix64 output function (Steele, Lea & Flood 2014).
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ULL;

__device__ __forceinline__ float act_f(float z, int act) {
  return act == 0 ? fmaxf(z, 0.0f) : z / (1.0f + expf(-z));
}
__device__ __forceinline__ float act_grad_f(float z, int act) {
  if (act == 0) return z > 0.0f ? 1.0f : 0.0f;
  float s = 1.0f / (1.0f + expf(-z));
  return s * (1.0f + z * (1.0f - s));
}
__device__ __forceinline__ float out_f(float z, int out_act) {
  return out_act == 0 ? z : (z > 20.0f ? z : log1pf(expf(z)));
}
__device__ __forceinline__ float out_grad_f(float z, int out_act) {
  return out_act == 0 ? 1.0f : 1.0f / (1.0f + expf(-z));
}

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace dinr
