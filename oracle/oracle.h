/*
 * FP64 CPU oracle for the dense (intrinsic x extrinsic) likelihood of the
 * sampler-free gravitational-wave method (arXiv 2507.16022).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA library and includes nothing from it.
 *
 * Complex arrays are interleaved (re, im) doubles.  Layouts:
 *   h      [I][M][B]   bank waveform components h_{i m}(f_b), d_L = d_L^0
 *   R      [E][D][M]   complex detector response of mode m
 *   t      [E][D]      arrival time at detector d (s)
 *   data   [D][B]      detector data d_d(f_b)
 *   psd    [D][B]      one-sided PSD S_d(f_b)
 *   f, w   [B]         bin frequencies and quadrature weights
 *   mode_m [M]         azimuthal number of each mode
 *
 * Inner product (Eq. inner_product): <a|b> = sum_d sum_b 4 w_b a b^* / S_d.
 * Log-likelihood (Eq. lnlike): ln L = Re<d|h> - <h|h>/2.
 */
#ifndef DOTPE_ORACLE_H
#define DOTPE_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct or_problem {
  int n_int, n_ext, n_det, n_modes, n_bins, n_phi;
  const int *mode_m;
  const double *f, *w, *psd, *data;  /* data: complex */
  const double *h;                   /* complex [I][M][B] */
  const double *R;                   /* complex [E][D][M] */
  const double *t;                   /* [E][D] */
  const double *ln_w_int, *ln_w_ext; /* [I], [E] (may be NULL: zeros) */
  double u_min;                      /* d_L^0 / d_max of pi(d_L) ~ d_L^2 */
  /* relative binning (App. A), both or neither (NULL: plain quadrature with w),
   * per component j (a mode, or the (mode, polarisation) pair j = m n_pol + p):
   * rb_dh complex [D][J][B] = W^{<d|h>}_{d j b}, rb_hh complex [D][J][J][B] =
   * W^{<h|h>}_{d j j' b} (J = M n_pol); then <d|h_j>_d = sum_b W^{<d|h>}_{d j b} h_j^*(f_b)
   * and <h_j|h_j'>_d = sum_b W^{<h|h>}_{d j j' b} h_j(f_b) h_j'^*(f_b) (Eqs. dh_weights,
   * hh_weights, d_h, h_h).  Route O2 only. */
  const double *rb_dh, *rb_hh;
  /* polarisation-resolved (precessing) bank (Sec. IV.A general case,
   * Eqs. dh_ieo, hh_ieo with the index p): n_pol = 2, h complex [I][M][2][B]
   * (h_{i m p}, p = +, x), F [E][D][2] real antenna patterns F_{e d p} replacing R:
   * the strain is sum_{m,p} F_{edp} h_{imp} e^{i m phi} T.  n_pol = 0 or 1: h [I][M][B]
   * and R as above. */
  int n_pol;
  const double *F;
} or_problem;

/* Per-(i,e) outputs. */
typedef struct or_pair_out {
  double lnl_marg;    /* ln Lbar_ie = ln( (1/N_phi) sum_o Lbar_ieo ), -inf if no phase passes */
  double lnl_sq;      /* ln sum_o Lbar_ieo^2 (for N_eff), -inf if none */
  double lnl_ml_max;  /* max_o ln L^ML_ieo */
  int32_t argmax_o;   /* phase index of lnl_ml_max (lowest on ties) */
  int32_t n_pass;     /* phases that passed the ML cut */
} or_pair_out;

typedef struct or_evidence_out {
  double ln_z;        /* Eq. Z_sum */
  double n_eff, n_eff_int, n_eff_ext; /* Eqs. posterior_element, int_ess, ext_ess */
  double max_lnl_ml;
  int64_t arg_i, arg_e, arg_o;
  int64_t n_marginalised;
} or_evidence_out;

/* Eq. inner_product folded into per-bin data weights:
 *   c_{d,b} = 4 w_b conj(d_d(f_b)) / S_d(f_b),  omega_{d,b} = 4 w_b / S_d(f_b). */
int or_data_weights(int D, int B, const double *w, const double *psd, const double *data,
                    double *c_out, double *omega_out);

/* Relative-binning weights (App. A, Eqs. dh_weights, hh_weights) on a fine
 * frequency grid ff[n] (increasing) with quadrature weights dff[n]:
 *   <a|b>_d = sum_n 4 dff_n a(f_n) b^*(f_n) / S_d(f_n),
 *   W^{<d|h>}_{d m b}    = <d_d | h0_dm s_b>_d / h0_dm^*(f_b)
 *   W^{<h|h>}_{d m m' b} = <h0_dm | h0_dm' s_b>_d / (h0_dm(f_b) h0_dm'^*(f_b))
 * with h0_dm(f) = h0_m(f) e^{-2 pi i f t0_d}, the reference waveform's modes
 * arriving at detector d at t0_d (constant factors such as the response
 * cancel in the ratios; the time shift does not), and s_b the piecewise-linear
 * hat functions on the nodes f_b = ff[node[b]] (s_b(f_b') = delta_bb',
 * supported on [f_{b-1}, f_{b+1}]; fine points outside [f_0, f_{B-1}] do not
 * enter).  psd, data: [D][n]; h0: complex [M][n]; t0: [D] (NULL: 0);
 * node: [B] increasing fine-grid indices.  w_dh: complex [D][M][B];
 * w_hh: complex [D][M][M][B].  Returns -1 if some |h0_m(f_b)| is 0. */
int or_rb_weights(int D, int M, int64_t n_fine, const double *ff, const double *dff, const double *psd,
                  const double *data, const double *h0, const double *t0, int B, const int64_t *node,
                  double *w_dh, double *w_hh);

/* Route O1 (plain definition): for one (i, e) build the detector strain of
 * Eq. h_k at d_L = d_L^0 and phase phi_o = 2 pi o / n_phi, then evaluate
 * Re<d|h> and <h|h> by the frequency sum.  dh_out, hh_out: [n_phi]. */
int or_direct_phases(const or_problem *p, int64_t i, int64_t e, double *dh_out, double *hh_out);

/* Route O2 (Eqs. dh_ieo, hh_ieo): per-mode components for one (i, e):
 *   z_m = sum_d R_{e,d,m} sum_b c_{d,b} e^{-2 pi i f_b t_{e,d}} h_{i m}(f_b)
 *   H_{m m'} = sum_d R_{e,d,m} R^*_{e,d,m'} <h_{i m}|h_{i m'}>_d
 * z_out: complex [M]; H_out: complex [M][M]. */
int or_mode_components(const or_problem *p, const double *c, const double *omega,
                       int64_t i, int64_t e, double *z_out, double *H_out);

/* Orbital-phase rotation (Phi_m = e^{i m phi}): dh_o = Re sum_m z_m e^{i m phi_o},
 * hh_o = Re sum_{m m'} H_{m m'} e^{i (m - m') phi_o}. */
int or_rotate_phases(int M, const int *mode_m, const double *z, const double *H, int n_phi,
                     double *dh_out, double *hh_out);

/* Eq. bestfit_lnl. */
double or_lnl_ml(double dh, double hh);

/* Eq. lnl_dist_marginalized with pi(d_L) = 3 d_L^2 / d_max^3 on (0, d_max],
 * u_min = d_L^0 / d_max: returns ln Lbar(dh, hh). */
double or_dist_marg(double dh, double hh, double u_min);

/* Distance draw of one posterior sample (App. C: distance drawn per pair from
 * the summand of the distance marginal): the conditional density of
 * u = d_L^0 / d_L on [u_min, inf) is proportional to u^-4 exp(dh u - hh u^2 / 2)
 * (pi(d_L) ~ d_L^2); returns d_L / d_L^0 = 1/u at cumulative probability q in
 * [0, 1), found by bisection on the adaptive Gauss-Kronrod CDF.  hh <= 0: the
 * prior, d_L / d_L^0 = (1 - q)^(1/3) / u_min. */
double or_dist_sample(double dh, double hh, double u_min, double q);

/* Full per-pair evaluation (route O2, phase grid, ML cut, distance marginal,
 * phase average) for an explicit list of pairs.  lnl_ml_threshold: phases
 * with ln L^ML below it are dropped (pass -INFINITY for no cut). */
int or_eval_pairs(const or_problem *p, int64_t n_pairs, const int64_t *pi, const int64_t *pe,
                  double lnl_ml_threshold, int n_threads, or_pair_out *out);

/* Same over the whole I x E grid (out: [I][E]); with cut_delta > 0 the
 * threshold is max_{ieo} ln L^ML - cut_delta (Eq. coherent_ML_selection),
 * found in a first pass.  Returns the threshold used via *thr_out. */
int or_eval_grid(const or_problem *p, double cut_delta, int n_threads, or_pair_out *out,
                 double *thr_out);

/* Route O1 over the whole grid (no distance marginal): max_o ln L^ML per pair. */
int or_direct_grid_ml(const or_problem *p, int n_threads, double *lnl_ml_max_out);

/* Evidence and effective sample sizes from per-pair outputs over the full
 * grid [I][E] (Eq. Z_sum with w_o = 1; Eqs. posterior_element, int_ess, ext_ess).
 * ln_p_int [I] and ln_p_ext [E] (may be NULL) receive ln sum_{e,o} p_ieo and
 * ln sum_{i,o} p_ieo. */
int or_evidence(const or_problem *p, const or_pair_out *grid, or_evidence_out *ev,
                double *ln_p_int, double *ln_p_ext);

/* ---- Incoherent single-detector pre-selection (Sec. IV.D, App. B) ----------
 * Each detector k alone: the polarisation amplitudes x_{k+}, x_{kx} are free
 * (App. B: sky position, distance and polarisation angle are degenerate for
 * one detector), time and orbital phase run over regular grids.
 *   h_{i m p}(f_b) = K_{i m p} h_{i m}(f_b)        polarisation p = (+, x)
 *   <d|h>_{i k o t p}  = Re sum_{m,b} c_{k b} e^{-2 pi i f_b t_{k t}} h_{i m p}(f_b) e^{i m phi_o}
 *   <h|h>_{i k o p p'} = Re sum_{m,m',b} omega_{k b} h_{i m p} h^*_{i m' p'} e^{i (m - m') phi_o}
 *   ln L^ML_{i k o t}  = 1/2 dh^T [hh]^+ dh          (Eqs. dh_itop, x_ML, single_det_ML)
 *   ln L^inco.ML_i     = sum_k max_{o,t} ln L^ML_{i k o t}
 * and a row is kept when ln L^inco.ML_i >= max_j ln L^inco.ML_j - delta.
 * The sign of the phase factor differs from App. B's e^{-i m phi}: the grid
 * phi_o = 2 pi o / n_phi is closed under phi -> -phi, so the maximum over o is
 * the same.  [hh]^+ is the inverse when det > PRESEL_RANK_TOL hh_{++} hh_{xx},
 * else the pseudo-inverse of the rank-one limit, hh / (hh_{++} + hh_{xx})^2. */
#define OR_PRESEL_RANK_TOL 1e-3

typedef struct or_presel {
  int n_int, n_det, n_modes, n_bins, n_t, n_phi;
  const int *mode_m;
  const double *f, *w, *psd, *data;  /* data: complex [D][B] */
  const double *h;                   /* complex [I][M][B], or [I][M][2][B] when n_pol = 2 */
  const double *pol;                 /* complex [I][M][2]: K_{i m +}, K_{i m x} (n_pol = 1) */
  const double *t_grid;              /* [D][n_t] arrival times at detector k (s) */
  const double *rb_dh, *rb_hh;       /* relative binning as in or_problem, or NULL: [D][J][B] and
                                        [D][J][J][B] with J = M (mode bank) or 2M (n_pol = 2,
                                        component j = 2m + p) */
  int n_pol;                         /* 2: polarisation-resolved bank, h_{i m p} read directly */
} or_presel_problem;

/* Eqs. x_ML, single_det_ML: max over real (x_+, x_x) of
 * dh_+ x_+ + dh_x x_x - (a x_+^2 + 2 b x_+ x_x + c x_x^2)/2, with
 * hh = [[a, b], [b, c]] positive semi-definite (pseudo-inverse reading above). */
double or_quad_ml(double dh_p, double dh_x, double a, double b, double c);

/* ln L^ML_{i k o t} of one row i and detector k over the whole grid:
 * ml_out [n_phi][n_t]. */
int or_presel_grid(const or_presel_problem *p, int64_t i, int k, double *ml_out);

/* Every row: ml_ik [I][D] = max_{o,t} ln L^ML_{i k o t}, arg_ot [I][D][2] its
 * (o, t) (lowest t, then lowest o, on ties), lnl_inco [I], keep [I] (0/1) for
 * the window delta; *thr_out = max - delta, *arg_out = the row of the maximum
 * (lowest on ties).  Any output pointer may be NULL except lnl_inco. */
int or_presel(const or_presel_problem *p, double delta, int n_threads, double *ml_ik, int32_t *arg_ot,
              double *lnl_inco, uint8_t *keep, double *thr_out, int64_t *arg_out);

/* Number of hardware threads the oracle will use by default. */
int or_default_threads(void);

#ifdef __cplusplus
}
#endif
#endif
