/* A plain C caller of the library (no Python, no CUDA headers): a uniform flow on a
 * periodic curvilinear box must stay uniform (free-stream preservation of the metric
 * terms) and keep its conservation totals, in both precision forms.  Host buffers only:
 * the library stages them.  Exit status 0 on success. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "jz.h"

#define CHECK(call)                                                         \
  do {                                                                      \
    int rc_ = (call);                                                       \
    if (rc_ != JZ_OK) {                                                     \
      fprintf(stderr, "%s failed (%d): %s\n", #call, rc_, jz_last_error()); \
      return 1;                                                             \
    }                                                                       \
  } while (0)

int main(void) {
  const int ni = 24, nj = 16, nk = 12;
  const long n = (long)ni * nj * nk;
  const double pi = 3.14159265358979323846;
  const double L[3] = {2.0 * pi, 1.5 * pi, 1.0 * pi};
  double* xyz = malloc(sizeof(double) * 3 * n);
  double* q = malloc(sizeof(double) * 5 * n);
  double* out = malloc(sizeof(double) * 5 * n);
  if (!xyz || !q || !out) return 1;
  /* smooth periodic distortion of a box */
  for (int k = 0; k < nk; ++k)
    for (int j = 0; j < nj; ++j)
      for (int i = 0; i < ni; ++i) {
        const long p = ((long)k * nj + j) * ni + i;
        const double s = (double)i / ni, t = (double)j / nj, u = (double)k / nk;
        const double w = 0.05 * sin(2 * pi * s) * sin(2 * pi * t) * sin(2 * pi * u);
        xyz[0 * n + p] = L[0] * (s + w);
        xyz[1 * n + p] = L[1] * (t + 0.5 * w);
        xyz[2 * n + p] = L[2] * (u - w);
      }
  double period[9] = {L[0], 0, 0, 0, L[1], 0, 0, 0, L[2]};
  /* uniform Mach 0.5 flow: rho = 1, p = 1/gamma */
  const double gamma = 1.4, u0 = 0.5, v0 = 0.1, w0 = -0.2;
  for (long p = 0; p < n; ++p) {
    q[0 * n + p] = 1.0;
    q[1 * n + p] = u0;
    q[2 * n + p] = v0;
    q[3 * n + p] = w0;
    q[4 * n + p] = (1.0 / gamma) / (gamma - 1.0) + 0.5 * (u0 * u0 + v0 * v0 + w0 * w0);
  }
  jz_grid* g = NULL;
  CHECK(jz_create_grid(ni, nj, nk, xyz, period, JZ_TOPO_PERIODIC, &g));
  CHECK(jz_compute_metrics(g));
  for (int form = 0; form < 2; ++form) {
    jz_params prm;
    memset(&prm, 0, sizeof prm);
    prm.gamma = gamma; prm.Pr = 0.72; prm.Pr_sgs = 0.9; prm.Re = 1e4; prm.mach_ref = 0.5;
    prm.T_ref_K = 288.15; prm.S1_K = 110.4; prm.C_s = 0.18; prm.kappa2 = 0.25; prm.kappa4 = 1.0 / 64;
    prm.sigma = 2.0 / 3.0; prm.cfl = 0.5; prm.jet_mach = 1.4; prm.theta_mom = 0.05;
    prm.strouhal[0] = 0.2; prm.strouhal[1] = 0.4; prm.strouhal[2] = 0.6; prm.strouhal[3] = 0.8;
    prm.precision = form == 0 ? JZ_PREC_FP64 : JZ_PREC_FP32FLUX;
    jz_solver* s = NULL;
    CHECK(jz_create(g, &prm, NULL, &s));
    CHECK(jz_set_state(s, q, 0.0));
    jz_step_stats st0, st;
    CHECK(jz_rk_step(s, 0, &st0));
    CHECK(jz_rk_step(s, 5, &st));
    CHECK(jz_get_state(s, out));
    double dev = 0.0, drift = 0.0;
    for (long p = 0; p < 5 * n; ++p) dev = fmax(dev, fabs(out[p] - q[p]));
    for (int m = 0; m < 5; ++m) drift = fmax(drift, fabs(st.totals[m] - st0.totals[m]) / fmax(fabs(st0.totals[m]), 1.0));
    /* FP64: round-off; FP32-flux: the form's flux rounding (conservation bound 1e-10) */
    const double tol = form == 0 ? 1e-12 : 1e-6, tol_tot = form == 0 ? 1e-12 : 1e-10;
    printf("%s: 5 steps, t = %.6e, max |Q - Q0| = %.3e, totals drift = %.3e\n",
           form == 0 ? "FP64" : "FP32-flux", st.t, dev, drift);
    if (!(dev <= tol) || !(drift <= tol_tot) || st.steps != 5) {
      fprintf(stderr, "free-stream or conservation check failed\n");
      return 1;
    }
    CHECK(jz_destroy(s));
  }
  CHECK(jz_destroy_grid(g));
  free(xyz);
  free(q);
  free(out);
  printf("C ABI example OK\n");
  return 0;
}
