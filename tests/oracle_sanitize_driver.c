/* Drives every entry point of the FP64 oracle on small random problems, for a
 * build with AddressSanitizer and UndefinedBehaviorSanitizer (test only: the
 * values are not checked here, the sanitizers check every access). */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "../oracle/oracle.h"

static uint64_t rng_state = 88172645463325252ull;
static double urand(void) {
  rng_state ^= rng_state << 13;
  rng_state ^= rng_state >> 7;
  rng_state ^= rng_state << 17;
  return (double)(rng_state >> 11) / 9007199254740992.0;
}
static double *arr(size_t n, double lo, double hi) {
  double *a = malloc(sizeof(double) * n);
  for (size_t k = 0; k < n; ++k) a[k] = lo + (hi - lo) * urand();
  return a;
}

static int run_problem(int n_pol, int with_rb) {
  const int I = 5, E = 4, D = 2, M = 3, B = 24, NP = 8;
  const int J = M * (n_pol == 2 ? 2 : 1);
  int mode_m[3] = {2, 3, 4};
  double *f = arr(B, 20.0, 400.0), *w = arr(B, 1.0, 2.0), *psd = arr(D * B, 0.5, 2.0);
  for (int b = 1; b < B; ++b) f[b] = f[b - 1] + 10.0;
  double *data = arr(2 * D * B, -1.0, 1.0), *h = arr(2 * (size_t)I * J * B, -1.0, 1.0);
  double *R = arr(2 * (size_t)E * D * M, -1.0, 1.0), *F = arr((size_t)E * D * 2, -1.0, 1.0);
  double *t = arr((size_t)E * D, -0.01, 0.01), *lwi = arr(I, -0.5, 0.5), *lwe = arr(E, -0.5, 0.5);
  double *rbd = with_rb ? arr(2 * (size_t)D * J * B, -1.0, 1.0) : NULL;
  double *rbh = with_rb ? arr(2 * (size_t)D * J * J * B, 0.1, 1.0) : NULL;
  or_problem p = {I, E, D, M, B, NP, mode_m, f, w, psd, data, h, R, t, lwi, lwe, 0.5, rbd, rbh, n_pol, F};
  or_pair_out *grid = malloc(sizeof(or_pair_out) * I * E);
  double thr = 0.0, *ml = malloc(sizeof(double) * I * E), lpi[5], lpe[4];
  or_evidence_out ev;
  int rc = or_eval_grid(&p, 5.0, 2, grid, &thr);
  rc |= or_eval_grid(&p, 0.0, 1, grid, &thr);
  rc |= or_evidence(&p, grid, &ev, lpi, lpe);
  if (!with_rb) rc |= or_direct_grid_ml(&p, 2, ml);
  int64_t pi[3] = {0, 2, 4}, pe[3] = {3, 1, 0};
  rc |= or_eval_pairs(&p, 3, pi, pe, -INFINITY, 1, grid);
  double *c = malloc(sizeof(double) * 2 * D * B), *om = malloc(sizeof(double) * D * B);
  rc |= or_data_weights(D, B, w, psd, data, c, om);
  double z[2 * 3], H[2 * 9], dh[NP], hh[NP];
  rc |= or_mode_components(&p, c, om, 1, 2, z, H);
  rc |= or_rotate_phases(M, mode_m, z, H, NP, dh, hh);
  if (!with_rb) rc |= or_direct_phases(&p, 3, 1, dh, hh);
  free(f); free(w); free(psd); free(data); free(h); free(R); free(F); free(t); free(lwi); free(lwe);
  free(rbd); free(rbh); free(grid); free(ml); free(c); free(om);
  return rc;
}

static int run_rb_weights(void) {
  const int D = 2, J = 6, B = 12;
  const int64_t N = 400;
  double *ff = arr(N, 0.0, 1.0), *dff = arr(N, 0.5, 1.0), *psd = arr(D * N, 0.5, 2.0);
  for (int64_t n = 0; n < N; ++n) ff[n] = 20.0 + 0.5 * (double)n;
  double *data = arr(2 * D * N, -1.0, 1.0), *h0 = arr(2 * J * N, 0.5, 1.0), t0[2] = {0.001, -0.002};
  int64_t node[12];
  for (int b = 0; b < B; ++b) node[b] = (int64_t)b * 33;
  double *wdh = malloc(sizeof(double) * 2 * D * J * B), *whh = malloc(sizeof(double) * 2 * D * J * J * B);
  int rc = or_rb_weights(D, J, N, ff, dff, psd, data, h0, t0, B, node, wdh, whh);
  free(ff); free(dff); free(psd); free(data); free(h0); free(wdh); free(whh);
  return rc;
}

static int run_presel(int n_pol, int with_rb) {
  const int I = 4, D = 2, M = 3, B = 20, NT = 5, NP = 6;
  int mode_m[3] = {1, 2, 4};
  double *f = arr(B, 20.0, 30.0), *w = arr(B, 1.0, 2.0), *psd = arr(D * B, 0.5, 2.0);
  for (int b = 1; b < B; ++b) f[b] = f[b - 1] + 12.0;
  double *data = arr(2 * D * B, -1.0, 1.0), *h = arr(2 * (size_t)I * M * 2 * B, -1.0, 1.0);
  double *pol = arr(2 * (size_t)I * M * 2, -1.0, 1.0), *tg = arr((size_t)D * NT, -0.01, 0.01);
  const int J = M * (n_pol == 2 ? 2 : 1);
  double *rbd = with_rb ? arr(2 * (size_t)D * J * B, -1.0, 1.0) : NULL;
  double *rbh = with_rb ? arr(2 * (size_t)D * J * J * B, 0.1, 1.0) : NULL;
  or_presel_problem p = {I, D, M, B, NT, NP, mode_m, f, w, psd, data, h, n_pol == 2 ? NULL : pol, tg,
                         rbd, rbh, n_pol};
  double ml[4 * 2], inco[4], thr, g[6 * 5];
  int32_t arg[4 * 2 * 2];
  uint8_t keep[4];
  int64_t arg_i;
  int rc = or_presel_grid(&p, 1, 1, g);
  rc |= or_presel(&p, 20.0, 2, ml, arg, inco, keep, &thr, &arg_i);
  (void)or_quad_ml(1.0, 2.0, 1.0, 0.999, 1.0);
  free(f); free(w); free(psd); free(data); free(h); free(pol); free(tg); free(rbd); free(rbh);
  return rc;
}

int main(void) {
  int rc = 0;
  double s = 0.0;
  for (int k = 0; k < 200; ++k) {
    const double dh = -5.0 + 40.0 * urand(), hh = 60.0 * urand(), u = 0.05 + 3.0 * urand();
    s += or_dist_marg(dh, hh, u) + or_lnl_ml(dh, hh) + or_dist_sample(dh, hh, u, urand());
  }
  rc |= run_problem(1, 0);
  rc |= run_problem(1, 1);
  rc |= run_problem(2, 0);
  rc |= run_problem(2, 1);
  rc |= run_rb_weights();
  rc |= run_presel(1, 0);
  rc |= run_presel(2, 0);
  rc |= run_presel(1, 1);
  rc |= run_presel(2, 1);
  rc |= or_default_threads() < 1;
  printf("oracle driver: rc=%d checksum=%.6g\n", rc, s);
  return rc != 0;
}
