/*
 * dinr_example.c - the C ABI of libdinr used from plain C (no CUDA headers):
 * train a small network on the parallel-beam projections of a static sphere
 * and report the loss.
 *
 * Build (from the repository root, after building libdinr.so):
 *   gcc -std=c11 -O2 include/dinr_example.c -I include \
 *       -L paper_2404_19075_b300 -ldinr -Wl,-rpath,$PWD/paper_2404_19075_b300 -lm \
 *       -o dinr_example
 *   ./dinr_example [steps]
 *
 * The measured data are exact: a ray at distance h from the centre of a
 * sphere of radius a and attenuation rho crosses it over 2 sqrt(a^2 - h^2)
 * (Sec. III: the projection is the line integral over the field of view).
 * Exit status 0 when the loss after training is below a tenth of the first
 * step's.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "dinr.h"

enum { VIEWS = 64, ROWS = 32, COLS = 32 };

static int check(dinr_status s, dinr_ctx *ctx, const char *what) {
  if (s == DINR_OK) return 0;
  fprintf(stderr, "%s failed (status %d): %s\n", what, (int)s, dinr_last_error(ctx));
  return 1;
}

int main(int argc, char **argv) {
  const int steps = argc > 1 ? atoi(argv[1]) : 300;
  const double pi = 3.14159265358979323846;
  static double angle[VIEWS], view_t[VIEWS];
  for (int k = 0; k < VIEWS; ++k) {
    angle[k] = pi * k / VIEWS;
    view_t[k] = (double)k / VIEWS;
  }
  dinr_geometry g = {0};
  g.beam = DINR_BEAM_PARALLEL;
  g.n_views = VIEWS;
  g.det_rows = ROWS;
  g.det_cols = COLS;
  g.view_angle = angle;
  g.view_time = view_t;
  g.det_pitch_u = 2.0 / COLS;  /* the detector spans the unit FOV cylinder */
  g.det_pitch_v = 2.0 / ROWS;
  g.det_off_u = -1.0;
  g.det_off_v = -1.0;
  g.fov_r = 1.0;
  g.fov_z0 = -1.0;
  g.fov_z1 = 1.0;
  g.t0 = 0.0;
  g.t1 = 1.0;
  g.samples_per_ray = 32;
  g.mu0 = 1.0;

  /* a centred sphere: the projection does not depend on the view */
  const double a = 0.5, rho = 0.8;
  float *proj = malloc(sizeof(float) * VIEWS * ROWS * COLS);
  if (!proj) return 1;
  for (int m = 0; m < VIEWS; ++m)
    for (int r = 0; r < ROWS; ++r)
      for (int c = 0; c < COLS; ++c) {
        const double u = g.det_off_u + (c + 0.5) * g.det_pitch_u;
        const double v = g.det_off_v + (r + 0.5) * g.det_pitch_v;
        const double h2 = u * u + v * v;
        proj[(m * ROWS + r) * COLS + c] =
            h2 < a * a ? (float)(2.0 * rho * sqrt(a * a - h2)) : 0.0f;
      }

  dinr_net net = {0};
  net.n_freq = 6;
  net.hidden_layers = 3;
  net.width = 64;
  net.act = DINR_ACT_RELU;
  net.out_act = DINR_OUT_SOFTPLUS;
  net.prec = DINR_PREC_BF16;
  net.seed = 2001;
  net.encoding = DINR_ENC_OCTAVE;

  dinr_train tr = {0};
  tr.batch_rays = 1024;
  tr.sampler_seed = 3001;

  dinr_ctx *ctx = NULL;
  if (check(dinr_create(&g, &net, &tr, proj, 0, NULL, &ctx), NULL, "dinr_create")) return 1;
  free(proj);

  float first = 0.0f, loss = 0.0f;
  for (int s = 0; s < steps; ++s) {
    /* the built-in sampler; the loss is read back every 50 steps only */
    const int report = s == 0 || (s + 1) % 50 == 0 || s + 1 == steps;
    if (check(dinr_train_step(ctx, NULL, tr.batch_rays, 0, report ? &loss : NULL), ctx,
              "dinr_train_step"))
      return 1;
    if (s == 0) first = loss;
    if (report) printf("step %4d  loss %.6f\n", s + 1, loss);
  }
  printf("parameters: %lld\n", (long long)dinr_param_count(net.n_freq, net.hidden_layers,
                                                           net.width));
  dinr_destroy(ctx);
  return loss < 0.1f * first ? 0 : 2;
}
