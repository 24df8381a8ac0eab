/*
 * FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Plain, slow, obviously correct restatement of the likelihood of
 * arXiv 2507.16022, Sec. III-IV:
 *   Eq. inner_product  <a|b> = 4 sum_k sum_f a b^* / S_k  df
 *   Eq. lnlike         ln L = Re<d|h> - <h|h>/2
 *   Eq. h_k            h_k = (d0/d) sum_m h_m R_{k m} T_k Phi_m
 *   Eqs. dh_ieo/hh_ieo per-mode components and phase factors
 *   Eq. bestfit_lnl    ML over distance
 *   Eq. lnl_dist_marginalized, Eq. coherent_ML_selection, Eq. Z_sum,
 *   Eqs. posterior_element, int_ess, ext_ess.
 * Everything is double precision; no blocking, fusion or reordering beyond
 * the definitions.
 */
#include "oracle.h"

#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

typedef double complex cplx;

static const double TWO_PI = 6.283185307179586476925286766559;

static inline cplx ld_c(const double *a, int64_t k) { return a[2 * k] + I * a[2 * k + 1]; }
static inline void st_c(double *a, int64_t k, cplx v) {
  a[2 * k] = creal(v);
  a[2 * k + 1] = cimag(v);
}

int or_default_threads(void) {
  long n = sysconf(_SC_NPROCESSORS_ONLN);
  return n > 0 ? (int)n : 1;
}

/* ------------------------------------------------------------------------ */
/* Eq. inner_product -> per-bin data weights                                 */
/* ------------------------------------------------------------------------ */
int or_data_weights(int D, int B, const double *w, const double *psd, const double *data,
                    double *c_out, double *omega_out) {
  for (int d = 0; d < D; ++d)
    for (int b = 0; b < B; ++b) {
      int64_t k = (int64_t)d * B + b;
      double om = 4.0 * w[b] / psd[k];
      if (omega_out) omega_out[k] = om;
      if (c_out) st_c(c_out, k, om * conj(ld_c(data, k)));
    }
  return 0;
}

/* Phi on the regular grid phi_o = 2 pi o / N_phi: e^{i k phi_o} with the integer
 * k o reduced modulo N_phi first, so that equal phases give equal values and
 * ties between grid points are exact. */
static cplx grid_phase(int k, int o, int n_phi) {
  long r = ((long)k * (long)o) % n_phi;
  if (r < 0) r += n_phi;
  return cexp(I * TWO_PI * (double)r / (double)n_phi);
}

/* Polarisations per mode (2 for a polarisation-resolved bank), the waveform
 * component h_{i m q}(f_b) and its response at detector d for sample e:
 * R_{e d m} (q = 0) or the real antenna pattern F_{e d q}. */
static inline int n_pol_of(const or_problem *p) { return p->n_pol == 2 ? 2 : 1; }
static inline cplx hval(const or_problem *p, int64_t i, int m, int q, int b) {
  const int NP = n_pol_of(p);
  return ld_c(p->h, ((i * p->n_modes + m) * NP + q) * (int64_t)p->n_bins + b);
}
static inline cplx resp(const or_problem *p, int64_t e, int d, int m, int q) {
  if (n_pol_of(p) == 2) return p->F[(e * p->n_det + d) * 2 + q];
  return ld_c(p->R, (e * p->n_det + d) * p->n_modes + m);
}

/* ------------------------------------------------------------------------ */
/* Relative-binning weights (App. A, Eqs. dh_weights, hh_weights)            */
/* ------------------------------------------------------------------------ */
/* hat function of node b at fine frequency f (nodes fn[0..B-1]) */
static double hat(const double *fn, int B, int b, double f) {
  if (b > 0 && f >= fn[b - 1] && f <= fn[b]) return (f - fn[b - 1]) / (fn[b] - fn[b - 1]);
  if (b < B - 1 && f >= fn[b] && f <= fn[b + 1]) return (fn[b + 1] - f) / (fn[b + 1] - fn[b]);
  return f == fn[b] ? 1.0 : 0.0;
}

int or_rb_weights(int D, int M, int64_t n_fine, const double *ff, const double *dff, const double *psd,
                  const double *data, const double *h0, const double *t0, int B, const int64_t *node,
                  double *w_dh, double *w_hh) {
  double *fn = malloc(sizeof(double) * (size_t)B);
  if (!fn) return -1;
  for (int b = 0; b < B; ++b) fn[b] = ff[node[b]];
  for (int m = 0; m < M; ++m)
    for (int b = 0; b < B; ++b)
      if (cabs(ld_c(h0, (int64_t)m * n_fine + node[b])) == 0.0) {
        free(fn);
        return -1;
      }
  for (int d = 0; d < D; ++d) {
    const double td = t0 ? t0[d] : 0.0;
    for (int b = 0; b < B; ++b) {
      /* the support of s_b: fine points from node b-1 to node b+1 */
      const int64_t n0 = node[b > 0 ? b - 1 : 0], n1 = node[b < B - 1 ? b + 1 : B - 1];
      const cplx Tb = cexp(-I * TWO_PI * fn[b] * td);
      for (int m = 0; m < M; ++m) {
        const cplx h0b = ld_c(h0, (int64_t)m * n_fine + node[b]) * Tb; /* h0_dm(f_b) */
        cplx acc = 0.0;
        for (int64_t n = n0; n <= n1; ++n) {
          const cplx h0n = ld_c(h0, (int64_t)m * n_fine + n) * cexp(-I * TWO_PI * ff[n] * td);
          acc += 4.0 * dff[n] * ld_c(data, (int64_t)d * n_fine + n) * conj(h0n) * hat(fn, B, b, ff[n]) /
                 psd[(int64_t)d * n_fine + n];
        }
        st_c(w_dh, ((int64_t)d * M + m) * B + b, acc / conj(h0b));
        for (int mp = 0; mp < M; ++mp) {
          const cplx h0pb = ld_c(h0, (int64_t)mp * n_fine + node[b]) * Tb;
          cplx a2 = 0.0;
          for (int64_t n = n0; n <= n1; ++n) {
            const cplx T = cexp(-I * TWO_PI * ff[n] * td);
            a2 += 4.0 * dff[n] * ld_c(h0, (int64_t)m * n_fine + n) * T * conj(ld_c(h0, (int64_t)mp * n_fine + n) * T) *
                  hat(fn, B, b, ff[n]) / psd[(int64_t)d * n_fine + n];
          }
          st_c(w_hh, (((int64_t)d * M + m) * M + mp) * B + b, a2 / (h0b * conj(h0pb)));
        }
      }
    }
  }
  free(fn);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Route O1: plain definition per (i, e, o)                                  */
/* ------------------------------------------------------------------------ */
int or_direct_phases(const or_problem *p, int64_t i, int64_t e, double *dh_out, double *hh_out) {
  const int M = p->n_modes, D = p->n_det, B = p->n_bins;
  for (int o = 0; o < p->n_phi; ++o) {
    double dh = 0.0, hh = 0.0;
    for (int d = 0; d < D; ++d) {
      double t = p->t[e * D + d];
      for (int b = 0; b < B; ++b) {
        /* strain of Eq. h_k at d_L = d_L^0 */
        cplx hk = 0.0;
        for (int m = 0; m < M; ++m) {
          cplx Phi = grid_phase(p->mode_m[m], o, p->n_phi);
          for (int q = 0; q < n_pol_of(p); ++q) hk += hval(p, i, m, q, b) * resp(p, e, d, m, q) * Phi;
        }
        hk *= cexp(-I * TWO_PI * p->f[b] * t);
        double wgt = 4.0 * p->w[b] / p->psd[(int64_t)d * B + b];
        cplx dk = ld_c(p->data, (int64_t)d * B + b);
        dh += wgt * creal(dk * conj(hk));
        hh += wgt * creal(hk * conj(hk));
      }
    }
    dh_out[o] = dh;
    hh_out[o] = hh;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Route O2: per-mode components, then phase rotation                        */
/* ------------------------------------------------------------------------ */
/* <h_{i m q}|h_{i m' q'}>_d = sum_b omega_{d b} h_{m q} h_{m' q'}^*  -> hm[d][M NP][M NP]
 * (index m NP + q; relative binning: the weight W^{<h|h>}_{d m m' q q' b} of each
 * pair of (mode, polarisation) components, Eqs. hh_weights and h_h, stored
 * [D][M NP][M NP][B] with the same component index) */
static void mode_overlaps(const or_problem *p, const double *omega, int64_t i, cplx *hm) {
  const int M = p->n_modes, D = p->n_det, B = p->n_bins, NP = n_pol_of(p), J = M * NP;
  for (int d = 0; d < D; ++d)
    for (int j = 0; j < J; ++j)
      for (int jp = 0; jp < J; ++jp) {
        const int m = j / NP, q = j % NP, mp = jp / NP, qp = jp % NP;
        cplx acc = 0.0;
        for (int b = 0; b < B; ++b) {
          cplx wgt = p->rb_hh ? ld_c(p->rb_hh, (((int64_t)d * J + j) * J + jp) * B + b)
                              : (cplx)omega[(int64_t)d * B + b];
          acc += wgt * hval(p, i, m, q, b) * conj(hval(p, i, mp, qp, b));
        }
        hm[((int64_t)d * J + j) * J + jp] = acc;
      }
}

/* Data weight of component (m, q) at bin b: c_{d b} = 4 w_b conj(d) / S (plain
 * quadrature), or (W^{<d|h>}_{d m q b})^* with relative binning (Eqs. dh_weights,
 * d_h: Re<d|h> = Re sum_b c h), stored [D][M NP][B] with index m NP + q. */
static cplx data_weight(const or_problem *p, const double *c, int d, int m, int q, int b) {
  const int NP = n_pol_of(p);
  if (p->rb_dh) return conj(ld_c(p->rb_dh, ((int64_t)d * p->n_modes * NP + m * NP + q) * p->n_bins + b));
  return ld_c(c, (int64_t)d * p->n_bins + b);
}

static void mode_components_cached(const or_problem *p, const double *c, const cplx *hm,
                                   int64_t i, int64_t e, cplx *z, cplx *H) {
  const int M = p->n_modes, D = p->n_det, B = p->n_bins, NP = n_pol_of(p), J = M * NP;
  for (int m = 0; m < M; ++m) z[m] = 0.0;
  for (int m = 0; m < M * M; ++m) H[m] = 0.0;
  for (int d = 0; d < D; ++d) {
    double t = p->t[e * D + d];
    /* <d_k | h_{m q} T_k> summed over b, i.e. sum_b c_{d b} T h_{m q} (real part taken later) */
    for (int m = 0; m < M; ++m)
      for (int q = 0; q < NP; ++q) {
        cplx acc = 0.0;
        for (int b = 0; b < B; ++b)
          acc += data_weight(p, c, d, m, q, b) * cexp(-I * TWO_PI * p->f[b] * t) * hval(p, i, m, q, b);
        z[m] += resp(p, e, d, m, q) * acc;
      }
    for (int m = 0; m < M; ++m)
      for (int mp = 0; mp < M; ++mp)
        for (int q = 0; q < NP; ++q)
          for (int qp = 0; qp < NP; ++qp)
            H[m * M + mp] += resp(p, e, d, m, q) * conj(resp(p, e, d, mp, qp)) *
                             hm[((int64_t)d * J + m * NP + q) * J + mp * NP + qp];
  }
}

int or_mode_components(const or_problem *p, const double *c, const double *omega, int64_t i,
                       int64_t e, double *z_out, double *H_out) {
  const int M = p->n_modes, D = p->n_det;
  const int J = M * n_pol_of(p);
  cplx *hm = malloc(sizeof(cplx) * (size_t)D * J * J);
  cplx *z = malloc(sizeof(cplx) * (size_t)M);
  cplx *H = malloc(sizeof(cplx) * (size_t)M * M);
  if (!hm || !z || !H) {
    free(hm); free(z); free(H);
    return -1;
  }
  mode_overlaps(p, omega, i, hm);
  mode_components_cached(p, c, hm, i, e, z, H);
  for (int m = 0; m < M; ++m) st_c(z_out, m, z[m]);
  for (int m = 0; m < M * M; ++m) st_c(H_out, m, H[m]);
  free(hm); free(z); free(H);
  return 0;
}

static void rotate(int M, const int *mode_m, const cplx *z, const cplx *H, int n_phi,
                   double *dh_out, double *hh_out) {
  for (int o = 0; o < n_phi; ++o) {
    cplx dh = 0.0, hh = 0.0;
    for (int m = 0; m < M; ++m) dh += z[m] * grid_phase(mode_m[m], o, n_phi);
    for (int m = 0; m < M; ++m)
      for (int mp = 0; mp < M; ++mp)
        hh += H[m * M + mp] * grid_phase(mode_m[m] - mode_m[mp], o, n_phi);
    dh_out[o] = creal(dh);
    hh_out[o] = creal(hh);
  }
}

int or_rotate_phases(int M, const int *mode_m, const double *z, const double *H, int n_phi,
                     double *dh_out, double *hh_out) {
  cplx *zz = malloc(sizeof(cplx) * (size_t)M);
  cplx *HH = malloc(sizeof(cplx) * (size_t)M * M);
  if (!zz || !HH) {
    free(zz); free(HH);
    return -1;
  }
  for (int m = 0; m < M; ++m) zz[m] = ld_c(z, m);
  for (int m = 0; m < M * M; ++m) HH[m] = ld_c(H, m);
  rotate(M, mode_m, zz, HH, n_phi, dh_out, hh_out);
  free(zz); free(HH);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Eq. bestfit_lnl                                                           */
/* ------------------------------------------------------------------------ */
double or_lnl_ml(double dh, double hh) {
  if (!(hh > 0.0) || !(dh > 0.0)) return 0.0;
  return dh * dh / (2.0 * hh);
}

/* ------------------------------------------------------------------------ */
/* Eq. lnl_dist_marginalized                                                  */
/*                                                                          */
/* Lbar = int_0^dmax 3 d^2/dmax^3 exp(dh u - hh u^2 / 2) dd,  u = d0/d.       */
/* With u = d0/d the prior measure is 3 u_min^3 u^-4 du on [u_min, inf), and  */
/* with v = sqrt(hh) u, x = dh/sqrt(hh), s = sqrt(hh) u_min:                  */
/*   Lbar = 3 s^3 e^{x^2/2} int_s^inf v^-4 e^{-(v-x)^2/2} dv.                 */
/* The integral is done by adaptive Gauss-Kronrod (7/15) on the log-shifted  */
/* integrand.                                                                */
/* ------------------------------------------------------------------------ */
/* Kronrod 15-point abscissae (positive half) and weights, with the embedded
 * 7-point Gauss weights (published tables; QUADPACK qk15). */
static const double XGK[8] = {
    0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
    0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
    0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
    0.207784955007898467600689403773245, 0.000000000000000000000000000000000};
static const double WGK[8] = {
    0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
    0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
    0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
    0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
static const double WG[4] = {0.129484966168869693270611432679082,
                             0.279705391489276667901467771423780,
                             0.381830050505118944950369775488975,
                             0.417959183673469387755102040816327};

typedef struct {
  double x, shift;
} dm_ctx;

/* integrand v^-4 e^{-(v-x)^2/2} divided by e^{shift} */
static inline double dm_f(const dm_ctx *c, double v) {
  double a = -4.0 * log(v) - 0.5 * (v - c->x) * (v - c->x) - c->shift;
  return exp(a);
}

static void gk15(const dm_ctx *c, double a, double b, double *res, double *err) {
  double cen = 0.5 * (a + b), hl = 0.5 * (b - a);
  double fc = dm_f(c, cen);
  double rk = fc * WGK[7], rg = fc * WG[3];
  for (int j = 0; j < 7; ++j) {
    double dx = hl * XGK[j];
    double f1 = dm_f(c, cen - dx), f2 = dm_f(c, cen + dx);
    rk += WGK[j] * (f1 + f2);
    if (j % 2 == 1) rg += WG[j / 2] * (f1 + f2);
  }
  *res = rk * hl;
  *err = fabs((rk - rg) * hl);
}

#define DM_MAXPANEL 2000
double or_dist_marg(double dh, double hh, double u_min) {
  if (!(hh > 0.0)) return 0.0; /* no signal power: likelihood ratio 1 at every distance */
  double r = sqrt(hh);
  double x = dh / r, s = r * u_min;
  if (!(s > 0.0)) return 0.0;
  /* phi(v) = -4 ln v - (v-x)^2/2 has, for x > 4, a local minimum at v1 and a
   * local maximum at v2 (roots of v^2 - x v + 4 = 0); its maximum on [s, inf)
   * is at s or at v2. */
  double v1 = -1.0, v2 = -1.0;
  if (x > 4.0) {
    double q = sqrt(x * x - 16.0);
    v1 = 0.5 * (x - q);
    v2 = 0.5 * (x + q);
  }
  double phis = -4.0 * log(s) - 0.5 * (s - x) * (s - x);
  double pmax = phis;
  if (v2 > s) {
    double phi2 = -4.0 * log(v2) - 0.5 * (v2 - x) * (v2 - x);
    if (phi2 > pmax) pmax = phi2;
  }
  dm_ctx c = {x, pmax};
  /* initial breakpoints: geometric from s, the stationary points, and a
   * ladder around the Gaussian peak; beyond hi the integrand is < e^-800 of
   * its maximum */
  double peak = (v2 > s) ? v2 : s;
  double hi = (x > s ? x : s) + 40.0;
  double bp[128];
  int nb = 0;
  bp[nb++] = s;
  for (double v = 2.0 * s; v < hi && nb < 40; v *= 2.0) bp[nb++] = v;
  if (v1 > s) bp[nb++] = v1;
  if (v2 > s) bp[nb++] = v2;
  const double ladder[] = {-16, -8, -4, -2, -1, -0.5, 0.5, 1, 2, 4, 8, 16};
  for (int k = 0; k < 12; ++k) {
    double v = peak + ladder[k];
    if (v > s && v < hi) bp[nb++] = v;
  }
  bp[nb++] = hi;
  /* sort breakpoints */
  for (int a = 1; a < nb; ++a)
    for (int b = a; b > 0 && bp[b] < bp[b - 1]; --b) {
      double tmp = bp[b];
      bp[b] = bp[b - 1];
      bp[b - 1] = tmp;
    }
  static __thread double pa[DM_MAXPANEL], pb[DM_MAXPANEL], pr[DM_MAXPANEL], pe[DM_MAXPANEL];
  int np = 0;
  double tot = 0.0, terr = 0.0;
  for (int k = 0; k + 1 < nb; ++k) {
    if (!(bp[k + 1] > bp[k])) continue;
    pa[np] = bp[k];
    pb[np] = bp[k + 1];
    gk15(&c, pa[np], pb[np], &pr[np], &pe[np]);
    tot += pr[np];
    terr += pe[np];
    ++np;
  }
  /* bisect the worst panel until the summed error estimate is small */
  while (terr > 1e-13 * fabs(tot) && np < DM_MAXPANEL - 1) {
    int w = 0;
    for (int k = 1; k < np; ++k)
      if (pe[k] > pe[w]) w = k;
    double a = pa[w], b = pb[w], mid = 0.5 * (a + b);
    if (!(mid > a && mid < b)) break;
    tot -= pr[w];
    terr -= pe[w];
    pa[w] = a; pb[w] = mid;
    gk15(&c, a, mid, &pr[w], &pe[w]);
    pa[np] = mid; pb[np] = b;
    gk15(&c, mid, b, &pr[np], &pe[np]);
    tot += pr[w] + pr[np];
    terr += pe[w] + pe[np];
    ++np;
    if (terr < 0.0) { /* recompute from scratch against cancellation drift */
      tot = 0.0; terr = 0.0;
      for (int k = 0; k < np; ++k) { tot += pr[k]; terr += pe[k]; }
    }
  }
  /* final sums from scratch */
  tot = 0.0;
  for (int k = 0; k < np; ++k) tot += pr[k];
  return 0.5 * x * x + log(3.0) + 3.0 * log(s) + pmax + log(tot);
}

/* integral of the log-shifted integrand over [a, b] by adaptive GK(7/15) */
static double dm_integral(const dm_ctx *c, double a, double b) {
  enum { NP = 512 };
  double pa[NP], pb[NP], pr[NP], pe[NP];
  int np = 1;
  pa[0] = a; pb[0] = b;
  gk15(c, a, b, &pr[0], &pe[0]);
  for (;;) {
    double tot = 0.0, err = 0.0;
    int w = 0;
    for (int k = 0; k < np; ++k) {
      tot += pr[k];
      err += pe[k];
      if (pe[k] > pe[w]) w = k;
    }
    if (err <= 1e-14 * fabs(tot) || np >= NP - 1) return tot;
    double mid = 0.5 * (pa[w] + pb[w]);
    if (!(mid > pa[w] && mid < pb[w])) return tot;
    pa[np] = mid; pb[np] = pb[w];
    pb[w] = mid;
    gk15(c, pa[w], pb[w], &pr[w], &pe[w]);
    gk15(c, pa[np], pb[np], &pr[np], &pe[np]);
    ++np;
  }
}

double or_dist_sample(double dh, double hh, double u_min, double q) {
  if (!(hh > 0.0)) return cbrt(1.0 - q) / u_min;
  const double r = sqrt(hh), x = dh / r, s = r * u_min;
  /* v = sqrt(hh) u: density ~ v^-4 e^{-(v-x)^2/2} on [s, inf); the shift is the
   * log-density's maximum (at s or at the local maximum v2 for x > 4) */
  double vmax = s, pmax = -4.0 * log(s) - 0.5 * (s - x) * (s - x);
  if (x > 4.0) {
    double v2 = 0.5 * (x + sqrt(x * x - 16.0));
    double p2 = -4.0 * log(v2) - 0.5 * (v2 - x) * (v2 - x);
    if (v2 > s && p2 > pmax) { pmax = p2; vmax = v2; }
  }
  dm_ctx c = {x, pmax};
  /* beyond max(s, x, vmax) + 40 the Gaussian factor is below e^-800 */
  double hi = fmax(fmax(s, x), vmax) + 40.0;
  double total = dm_integral(&c, s, hi);
  double lo = s, up = hi;
  for (int it = 0; it < 200 && up - lo > 1e-14 * up; ++it) {
    double mid = 0.5 * (lo + up);
    if (dm_integral(&c, s, mid) < q * total) lo = mid;
    else up = mid;
  }
  return r / (0.5 * (lo + up)); /* d/d0 = 1/u = sqrt(hh) / v */
}

/* ------------------------------------------------------------------------ */
/* Per-pair evaluation                                                       */
/* ------------------------------------------------------------------------ */
static double lse2(double a, double b) {
  if (a == -INFINITY) return b;
  if (b == -INFINITY) return a;
  double m = a > b ? a : b;
  return m + log(exp(a - m) + exp(b - m));
}

typedef struct {
  const or_problem *p;
  const double *c, *omega;
  int64_t n_pairs;
  const int64_t *pi, *pe;
  int64_t grid_e; /* >0: grid mode, pair k -> (k / grid_e, k % grid_e) */
  double thr;
  int mode; /* 0: max lnL^ML only, 1: full */
  or_pair_out *out;
  double *ml_out;
  int64_t k0, k1;
  double local_max;
} or_job;

static void pair_eval(const or_problem *p, const double *c, const cplx *hm, int64_t i, int64_t e,
                      double thr, int full, or_pair_out *o, double *dh, double *hh, cplx *z,
                      cplx *H) {
  mode_components_cached(p, c, hm, i, e, z, H);
  rotate(p->n_modes, p->mode_m, z, H, p->n_phi, dh, hh);
  double best = -INFINITY;
  int arg = 0;
  for (int q = 0; q < p->n_phi; ++q) {
    double l = or_lnl_ml(dh[q], hh[q]);
    if (l > best) { best = l; arg = q; }
  }
  o->lnl_ml_max = best;
  o->argmax_o = arg;
  if (!full) return;
  /* Eq. coherent_ML_selection, then Eq. lnl_dist_marginalized per phase and
   * the phase average with w_o = 1 */
  double s1 = -INFINITY, s2 = -INFINITY;
  int npass = 0;
  for (int q = 0; q < p->n_phi; ++q) {
    if (!(or_lnl_ml(dh[q], hh[q]) >= thr)) continue;
    double l = or_dist_marg(dh[q], hh[q], p->u_min);
    s1 = lse2(s1, l);
    s2 = lse2(s2, 2.0 * l);
    ++npass;
  }
  o->lnl_marg = (s1 == -INFINITY) ? -INFINITY : s1 - log((double)p->n_phi);
  o->lnl_sq = s2;
  o->n_pass = npass;
}

static void *job_run(void *arg) {
  or_job *j = (or_job *)arg;
  const or_problem *p = j->p;
  const int M = p->n_modes, D = p->n_det, np = p->n_phi;
  const int J = M * n_pol_of(p);
  cplx *hm = malloc(sizeof(cplx) * (size_t)D * J * J);
  cplx *z = malloc(sizeof(cplx) * (size_t)M);
  cplx *H = malloc(sizeof(cplx) * (size_t)M * M);
  double *dh = malloc(sizeof(double) * (size_t)np);
  double *hh = malloc(sizeof(double) * (size_t)np);
  int64_t cached_i = -1;
  double lmax = -INFINITY;
  for (int64_t k = j->k0; k < j->k1; ++k) {
    int64_t i, e;
    if (j->grid_e > 0) {
      i = k / j->grid_e;
      e = k % j->grid_e;
    } else {
      i = j->pi[k];
      e = j->pe[k];
    }
    if (i != cached_i) {
      mode_overlaps(p, j->omega, i, hm);
      cached_i = i;
    }
    or_pair_out tmp;
    or_pair_out *o = j->out ? &j->out[k] : &tmp;
    pair_eval(p, j->c, hm, i, e, j->thr, j->mode, o, dh, hh, z, H);
    if (j->ml_out) j->ml_out[k] = o->lnl_ml_max;
    if (o->lnl_ml_max > lmax) lmax = o->lnl_ml_max;
  }
  j->local_max = lmax;
  free(hm); free(z); free(H); free(dh); free(hh);
  return NULL;
}

static int run_jobs(const or_problem *p, int64_t n, const int64_t *pi, const int64_t *pe,
                    int64_t grid_e, double thr, int mode, int n_threads, or_pair_out *out,
                    double *ml_out, double *gmax) {
  const int D = p->n_det, B = p->n_bins;
  double *c = malloc(sizeof(double) * 2 * (size_t)D * B);
  double *om = malloc(sizeof(double) * (size_t)D * B);
  if (!c || !om) {
    free(c); free(om);
    return -1;
  }
  or_data_weights(D, B, p->w, p->psd, p->data, c, om);
  if (n_threads <= 0) n_threads = or_default_threads();
  if (n_threads > 256) n_threads = 256;
  if ((int64_t)n_threads > n) n_threads = n > 0 ? (int)n : 1;
  or_job jobs[256];
  pthread_t th[256];
  for (int t = 0; t < n_threads; ++t) {
    or_job *j = &jobs[t];
    memset(j, 0, sizeof(*j));
    j->p = p; j->c = c; j->omega = om;
    j->n_pairs = n; j->pi = pi; j->pe = pe; j->grid_e = grid_e;
    j->thr = thr; j->mode = mode; j->out = out; j->ml_out = ml_out;
    j->k0 = n * t / n_threads;
    j->k1 = n * (t + 1) / n_threads;
  }
  for (int t = 1; t < n_threads; ++t) pthread_create(&th[t], NULL, job_run, &jobs[t]);
  job_run(&jobs[0]);
  for (int t = 1; t < n_threads; ++t) pthread_join(th[t], NULL);
  double m = -INFINITY;
  for (int t = 0; t < n_threads; ++t)
    if (jobs[t].local_max > m) m = jobs[t].local_max;
  if (gmax) *gmax = m;
  free(c); free(om);
  return 0;
}

int or_eval_pairs(const or_problem *p, int64_t n_pairs, const int64_t *pi, const int64_t *pe,
                  double thr, int n_threads, or_pair_out *out) {
  return run_jobs(p, n_pairs, pi, pe, 0, thr, 1, n_threads, out, NULL, NULL);
}

int or_eval_grid(const or_problem *p, double cut_delta, int n_threads, or_pair_out *out,
                 double *thr_out) {
  int64_t n = (int64_t)p->n_int * p->n_ext;
  double thr = -INFINITY;
  if (cut_delta > 0.0) {
    double gmax;
    if (run_jobs(p, n, NULL, NULL, p->n_ext, -INFINITY, 0, n_threads, NULL, NULL, &gmax))
      return -1;
    thr = gmax - cut_delta;
  }
  if (thr_out) *thr_out = thr;
  return run_jobs(p, n, NULL, NULL, p->n_ext, thr, 1, n_threads, out, NULL, NULL);
}

typedef struct {
  const or_problem *p;
  double *out;
  int64_t k0, k1;
} o1_job;

static void *o1_run(void *arg) {
  o1_job *j = (o1_job *)arg;
  const or_problem *p = j->p;
  double *dh = malloc(sizeof(double) * (size_t)p->n_phi);
  double *hh = malloc(sizeof(double) * (size_t)p->n_phi);
  for (int64_t k = j->k0; k < j->k1; ++k) {
    int64_t i = k / p->n_ext, e = k % p->n_ext;
    or_direct_phases(p, i, e, dh, hh);
    double best = -INFINITY;
    for (int q = 0; q < p->n_phi; ++q) {
      double l = or_lnl_ml(dh[q], hh[q]);
      if (l > best) best = l;
    }
    j->out[k] = best;
  }
  free(dh); free(hh);
  return NULL;
}

int or_direct_grid_ml(const or_problem *p, int n_threads, double *out) {
  int64_t n = (int64_t)p->n_int * p->n_ext;
  if (n_threads <= 0) n_threads = or_default_threads();
  if (n_threads > 256) n_threads = 256;
  o1_job jobs[256];
  pthread_t th[256];
  for (int t = 0; t < n_threads; ++t) {
    jobs[t].p = p; jobs[t].out = out;
    jobs[t].k0 = n * t / n_threads;
    jobs[t].k1 = n * (t + 1) / n_threads;
  }
  for (int t = 1; t < n_threads; ++t) pthread_create(&th[t], NULL, o1_run, &jobs[t]);
  o1_run(&jobs[0]);
  for (int t = 1; t < n_threads; ++t) pthread_join(th[t], NULL);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Eq. Z_sum and the effective sample sizes                                   */
/* ------------------------------------------------------------------------ */
static double lse_array(const double *a, int64_t n, int64_t stride) {
  double m = -INFINITY;
  for (int64_t k = 0; k < n; ++k)
    if (a[k * stride] > m) m = a[k * stride];
  if (m == -INFINITY) return -INFINITY;
  double s = 0.0;
  for (int64_t k = 0; k < n; ++k) s += exp(a[k * stride] - m);
  return m + log(s);
}

int or_evidence(const or_problem *p, const or_pair_out *g, or_evidence_out *ev,
                double *ln_p_int, double *ln_p_ext) {
  const int64_t NI = p->n_int, NE = p->n_ext;
  const double ln_nphi = log((double)p->n_phi);
  /* ln p_ie summed over phases: ln(w_i w_e sum_o Lbar_ieo) */
  double *lp = malloc(sizeof(double) * (size_t)(NI * NE));
  double *lp2 = malloc(sizeof(double) * (size_t)(NI * NE));
  double *row = malloc(sizeof(double) * (size_t)NI);
  double *col = malloc(sizeof(double) * (size_t)NE);
  if (!lp || !lp2 || !row || !col) {
    free(lp); free(lp2); free(row); free(col);
    return -1;
  }
  double best = -INFINITY;
  int64_t bi = 0, be = 0, bo = 0, nmarg = 0;
  for (int64_t i = 0; i < NI; ++i)
    for (int64_t e = 0; e < NE; ++e) {
      const or_pair_out *o = &g[i * NE + e];
      double lw = (p->ln_w_int ? p->ln_w_int[i] : 0.0) + (p->ln_w_ext ? p->ln_w_ext[e] : 0.0);
      lp[i * NE + e] = (o->lnl_marg == -INFINITY) ? -INFINITY : lw + o->lnl_marg + ln_nphi;
      lp2[i * NE + e] = (o->lnl_sq == -INFINITY) ? -INFINITY : 2.0 * lw + o->lnl_sq;
      if (o->lnl_ml_max > best) { /* lexicographically lowest (i, e, o) on ties */
        best = o->lnl_ml_max;
        bi = i; be = e; bo = o->argmax_o;
      }
      nmarg += o->n_pass;
    }
  /* Z = 1/(N_i N_e N_phi) sum_ieo w_i w_e Lbar_ieo */
  double ls1 = lse_array(lp, NI * NE, 1);
  double ls2 = lse_array(lp2, NI * NE, 1);
  ev->ln_z = ls1 - log((double)NI) - log((double)NE) - ln_nphi;
  ev->n_eff = (ls1 == -INFINITY) ? 0.0 : exp(2.0 * ls1 - ls2);
  for (int64_t i = 0; i < NI; ++i) row[i] = lse_array(lp + i * NE, NE, 1);
  for (int64_t e = 0; e < NE; ++e) col[e] = lse_array(lp + e, NI, NE);
  double *row2 = malloc(sizeof(double) * (size_t)NI);
  double *col2 = malloc(sizeof(double) * (size_t)NE);
  for (int64_t i = 0; i < NI; ++i) row2[i] = 2.0 * row[i];
  for (int64_t e = 0; e < NE; ++e) col2[e] = 2.0 * col[e];
  double lr = lse_array(row2, NI, 1), lc = lse_array(col2, NE, 1);
  ev->n_eff_int = (ls1 == -INFINITY) ? 0.0 : exp(2.0 * ls1 - lr);
  ev->n_eff_ext = (ls1 == -INFINITY) ? 0.0 : exp(2.0 * ls1 - lc);
  ev->max_lnl_ml = best;
  ev->arg_i = bi; ev->arg_e = be; ev->arg_o = bo;
  ev->n_marginalised = nmarg;
  if (ln_p_int) memcpy(ln_p_int, row, sizeof(double) * (size_t)NI);
  if (ln_p_ext) memcpy(ln_p_ext, col, sizeof(double) * (size_t)NE);
  free(lp); free(lp2); free(row); free(col); free(row2); free(col2);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Incoherent single-detector pre-selection (Sec. IV.D, App. B)             */
/* ------------------------------------------------------------------------ */
/* Eqs. x_ML, single_det_ML: x^ML = hh^+ dh, ln L^ML = dh^T hh^+ dh / 2. */
double or_quad_ml(double dp, double dx, double a, double b, double c) {
  if (!(a > 0.0) && !(c > 0.0)) return 0.0; /* no template power: nothing to fit */
  double det = a * c - b * b;
  if (det > OR_PRESEL_RANK_TOL * a * c) return 0.5 * (c * dp * dp - 2.0 * b * dp * dx + a * dx * dx) / det;
  /* rank one: hh = lambda v v^T with lambda = a + c, hh^+ = hh / lambda^2 */
  double s = a + c;
  return 0.5 * (a * dp * dp + 2.0 * b * dp * dx + c * dx * dx) / (s * s);
}

/* Number of data-weight components per mode: 2 with relative binning of a
 * polarisation-resolved bank (one weight per (m, p), App. A's Eqs. dh_weights and
 * hh_weights with the component index j = 2m + p), else 1. */
static inline int presel_nw(const or_presel_problem *p) { return (p->rb_dh && p->n_pol == 2) ? 2 : 1; }

/* W_{j t b} = c_{k j b} T_{t k b} of one detector: [M nw][n_t][B] (Eq. dh_itop without
 * the waveform), c_{k j b} = 4 w_b d_k^*(f_b) / S_k(f_b) for every component, or
 * (W^{<d|h>}_{k j b})^* with relative binning (App. A), j = m for a mode bank (the
 * polarisation factors cancel in Eq. dh_weights for a reference h0_{mp} = K_{mp} h0_m)
 * and j = 2m + p for a polarisation-resolved bank. */
static cplx *presel_weights(const or_presel_problem *p, int k) {
  const int B = p->n_bins, NT = p->n_t, J = p->n_modes * presel_nw(p);
  const int64_t kb = (int64_t)k * B;
  cplx *W = malloc(sizeof(cplx) * (size_t)J * NT * B);
  if (!W) return NULL;
  for (int j = 0; j < J; ++j)
    for (int t = 0; t < NT; ++t) {
      double tt = p->t_grid[(int64_t)k * NT + t];
      for (int b = 0; b < B; ++b) {
        cplx c = p->rb_dh ? conj(ld_c(p->rb_dh, ((int64_t)k * J + j) * B + b))
                          : (4.0 * p->w[b] / p->psd[kb + b]) * conj(ld_c(p->data, kb + b));
        W[((int64_t)j * NT + t) * B + b] = c * cexp(-I * TWO_PI * p->f[b] * tt);
      }
    }
  return W;
}

static int presel_grid_w(const or_presel_problem *p, const cplx *W, int64_t i, int k, double *ml_out) {
  const int M = p->n_modes, B = p->n_bins, NT = p->n_t, NP = p->n_phi;
  const int nw = presel_nw(p), J = M * nw; /* weight component of (m, q): m nw + q (nw - 1) */
  const int64_t kb = (int64_t)k * B;
  cplx *hp = malloc(sizeof(cplx) * (size_t)2 * M * B); /* h_{i m p}(f_b): [p][m][b] */
  cplx *z = malloc(sizeof(cplx) * (size_t)2 * M);      /* [p][m]: sum_b W_{t b} h_{i m p}(f_b) */
  cplx *ov = malloc(sizeof(cplx) * (size_t)3 * M * M); /* [pp'][m][m']: sum_b omega h_{m p} h^*_{m' p'} */
  double *hh = malloc(sizeof(double) * (size_t)3 * NP); /* (++, +x, xx) per o */
  if (!hp || !z || !ov || !hh) {
    free(hp); free(z); free(ov); free(hh);
    return -1;
  }
  /* h_{i m p}: K_{i m p} h_{i m} for a mode bank, the bank's own polarisations
   * for a polarisation-resolved one (App. B's general form) */
  for (int q = 0; q < 2; ++q)
    for (int m = 0; m < M; ++m) {
      if (p->n_pol == 2) {
        for (int b = 0; b < B; ++b) hp[((int64_t)q * M + m) * B + b] = ld_c(p->h, ((i * M + m) * 2 + q) * B + b);
      } else {
        cplx K = ld_c(p->pol, (i * M + m) * 2 + q);
        for (int b = 0; b < B; ++b) hp[((int64_t)q * M + m) * B + b] = K * ld_c(p->h, (i * M + m) * B + b);
      }
    }
  /* <h|h>_{i k o p p'}: frequency sums per mode pair, then the phase factors */
  const int pq[3][2] = {{0, 0}, {0, 1}, {1, 1}};
  for (int r = 0; r < 3; ++r)
    for (int m = 0; m < M; ++m)
      for (int mp = 0; mp < M; ++mp) {
        cplx s = 0.0;
        for (int b = 0; b < B; ++b) {
          const int j = m * nw + pq[r][0] * (nw - 1), jp = mp * nw + pq[r][1] * (nw - 1);
          cplx wgt = p->rb_hh ? ld_c(p->rb_hh, (((int64_t)k * J + j) * J + jp) * B + b)
                              : (cplx)(4.0 * p->w[b] / p->psd[kb + b]);
          s += wgt * hp[((int64_t)pq[r][0] * M + m) * B + b] * conj(hp[((int64_t)pq[r][1] * M + mp) * B + b]);
        }
        ov[(r * M + m) * M + mp] = s;
      }
  for (int o = 0; o < NP; ++o)
    for (int r = 0; r < 3; ++r) {
      cplx acc = 0.0;
      for (int m = 0; m < M; ++m)
        for (int mp = 0; mp < M; ++mp)
          acc += ov[(r * M + m) * M + mp] * grid_phase(p->mode_m[m] - p->mode_m[mp], o, NP);
      hh[3 * o + r] = creal(acc);
    }
  /* <d|h>_{i k o t p} (Eq. dh_itop) and ln L^ML (Eq. single_det_ML) */
  for (int t = 0; t < NT; ++t) {
    for (int q = 0; q < 2; ++q)
      for (int m = 0; m < M; ++m) {
        cplx acc = 0.0;
        const int j = m * nw + q * (nw - 1);
        for (int b = 0; b < B; ++b) acc += W[((int64_t)j * NT + t) * B + b] * hp[((int64_t)q * M + m) * B + b];
        z[q * M + m] = acc;
      }
    for (int o = 0; o < NP; ++o) {
      double dh[2];
      for (int q = 0; q < 2; ++q) {
        cplx s = 0.0;
        for (int m = 0; m < M; ++m) s += z[q * M + m] * grid_phase(p->mode_m[m], o, NP);
        dh[q] = creal(s);
      }
      ml_out[(int64_t)o * NT + t] = or_quad_ml(dh[0], dh[1], hh[3 * o], hh[3 * o + 1], hh[3 * o + 2]);
    }
  }
  free(hp); free(z); free(ov); free(hh);
  return 0;
}

int or_presel_grid(const or_presel_problem *p, int64_t i, int k, double *ml_out) {
  cplx *W = presel_weights(p, k);
  if (!W) return -1;
  int rc = presel_grid_w(p, W, i, k, ml_out);
  free(W);
  return rc;
}

typedef struct {
  const or_presel_problem *p;
  int64_t r0, r1;
  double *ml_ik;
  int32_t *arg_ot;
  double *inco;
  cplx **W; /* per detector */
  int err;
} ps_job;

static void *ps_run(void *arg) {
  ps_job *j = (ps_job *)arg;
  const or_presel_problem *p = j->p;
  const int D = p->n_det, NT = p->n_t, NP = p->n_phi;
  double *g = malloc(sizeof(double) * (size_t)NP * NT);
  if (!g) {
    j->err = -1;
    return NULL;
  }
  for (int64_t i = j->r0; i < j->r1; ++i) {
    double sum = 0.0;
    for (int k = 0; k < D; ++k) {
      if (presel_grid_w(p, j->W[k], i, k, g)) {
        j->err = -1;
        free(g);
        return NULL;
      }
      double best = -INFINITY;
      int bo = 0, bt = 0;
      for (int t = 0; t < NT; ++t) /* lowest t, then lowest o, on ties */
        for (int o = 0; o < NP; ++o)
          if (g[(int64_t)o * NT + t] > best) {
            best = g[(int64_t)o * NT + t];
            bo = o;
            bt = t;
          }
      if (j->ml_ik) j->ml_ik[i * D + k] = best;
      if (j->arg_ot) {
        j->arg_ot[(i * D + k) * 2] = bo;
        j->arg_ot[(i * D + k) * 2 + 1] = bt;
      }
      sum += best;
    }
    j->inco[i] = sum;
  }
  free(g);
  return NULL;
}

int or_presel(const or_presel_problem *p, double delta, int n_threads, double *ml_ik, int32_t *arg_ot,
              double *lnl_inco, uint8_t *keep, double *thr_out, int64_t *arg_out) {
  const int64_t n = p->n_int;
  if (!lnl_inco) return -1;
  if (n_threads <= 0) n_threads = or_default_threads();
  if (n_threads > 256) n_threads = 256;
  if ((int64_t)n_threads > n) n_threads = n > 0 ? (int)n : 1;
  cplx *W[64];
  if (p->n_det < 1 || p->n_det > 64) return -1;
  for (int k = 0; k < p->n_det; ++k) W[k] = presel_weights(p, k);
  for (int k = 0; k < p->n_det; ++k)
    if (!W[k]) {
      for (int q = 0; q < p->n_det; ++q) free(W[q]);
      return -1;
    }
  ps_job jobs[256];
  pthread_t th[256];
  for (int t = 0; t < n_threads; ++t) {
    ps_job *j = &jobs[t];
    memset(j, 0, sizeof(*j));
    j->p = p;
    j->W = W;
    j->ml_ik = ml_ik;
    j->arg_ot = arg_ot;
    j->inco = lnl_inco;
    j->r0 = n * t / n_threads;
    j->r1 = n * (t + 1) / n_threads;
  }
  for (int t = 1; t < n_threads; ++t) pthread_create(&th[t], NULL, ps_run, &jobs[t]);
  ps_run(&jobs[0]);
  for (int t = 1; t < n_threads; ++t) pthread_join(th[t], NULL);
  for (int k = 0; k < p->n_det; ++k) free(W[k]);
  for (int t = 0; t < n_threads; ++t)
    if (jobs[t].err) return -1;
  /* Sec. IV.D selection: keep ln L^inco.ML_i >= max_j ln L^inco.ML_j - delta */
  double best = -INFINITY;
  int64_t bi = 0;
  for (int64_t i = 0; i < n; ++i)
    if (lnl_inco[i] > best) {
      best = lnl_inco[i];
      bi = i;
    }
  double thr = best - delta;
  if (keep)
    for (int64_t i = 0; i < n; ++i) keep[i] = lnl_inco[i] >= thr;
  if (thr_out) *thr_out = thr;
  if (arg_out) *arg_out = bi;
  return 0;
}
