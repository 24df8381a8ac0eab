/*
 * dotpe -- dense (intrinsic x extrinsic) gravitational-wave likelihood on one
 * GB300 GPU (sm_103a), after arXiv 2507.16022 ("Sampler-free gravitational
 * wave inference using matrix multiplication").
 *
 * C ABI.  Every function returns an int status: DOTPE_OK (0) or a negative
 * DOTPE_E_* code; dotpe_strerror() names the code and
 * dotpe_last_error_message() (thread-local) gives the detail of the last
 * failure on the calling thread.  No C++ exception crosses this boundary.
 * A dotpe_ctx may be used from several host threads; calls are serialised
 * internally.
 *
 * Pointers marked "host or device" are classified with
 * cudaPointerGetAttributes: device (or managed) pointers are read on the GPU,
 * anything else is read from host memory.  The library never keeps a
 * caller's pointer after the call returns: inputs are copied into memory the
 * context owns.  Complex arrays are interleaved (re, im) doubles.
 *
 * Notation (paper Sec. IV): i = intrinsic sample (bank row), e = extrinsic
 * sample, d = detector, m = azimuthal mode, b = frequency bin, o = phase
 * index of the regular grid phi_o = 2 pi o / N_phi (w_o = 1, Sec. IV.B).
 */
#ifndef DOTPE_H
#define DOTPE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DOTPE_ABI_VERSION 7

/* ---- status codes ------------------------------------------------------ */
#define DOTPE_OK 0
#define DOTPE_E_INVALID -1     /* bad argument, shape, NaN/Inf input, unknown id */
#define DOTPE_E_NOMEM -2       /* device or pinned host allocation failed */
#define DOTPE_E_ADMISSION -3   /* event can never fit the context's HBM budget */
#define DOTPE_E_NOT_READY -4   /* event not finished yet */
#define DOTPE_E_TIMEOUT -5     /* a bounded wait (host or device) ran out */
#define DOTPE_E_DEVICE -6      /* CUDA error; the context may be unusable */
#define DOTPE_E_NOT_FOUND -7   /* unknown bank or event id */
#define DOTPE_E_UNSUPPORTED -8 /* valid request this build does not serve */

/* ---- enums ------------------------------------------------------------- */
/* Arithmetic of the <d|h> GEMM (Eq. dh_ieo).  All accumulate in FP32.
 *   FP32   : SIMT FFMA path (the plain baseline)
 *   BF16   : one tcgen05 pass, bf16 operands
 *   FP16   : one tcgen05 pass, fp16 operands
 *   BF16X3 : split precision x = hi + lo (both bf16); hi*hi + hi*lo + lo*hi
 *   FP16X3 : the same split with fp16 hi and lo (operands scaled by powers of
 *            two to |x| <= 1; lo keeps ~2^-24 absolute accuracy)
 *   MIXED  : every pair screened with one fp16 pass (best ln L^ML only), then
 *            the tiles of 128 x 32 pairs that can reach the coherent-ML cut
 *            (Eq. coherent_ML_selection) recomputed in FP16X3 with the full
 *            marginalisation.  The screening margin is 2u (ml + sqrt(2 ml)
 *            sqrt<d|d>), u = 2^-11, around both the tile's and the global best
 *            ln L^ML; the cut is applied at (screened max - margin) - cut_delta.
 *            With the cut off, tiles more than 30 + 2 margins below the maximum
 *            keep their single-pass fp16 values (each of their pairs weighs
 *            < e^-30 of the best one). */
enum {
  DOTPE_PREC_FP32 = 0,
  DOTPE_PREC_BF16 = 1,
  DOTPE_PREC_FP16 = 2,
  DOTPE_PREC_BF16X3 = 3,
  DOTPE_PREC_FP16X3 = 4,
  DOTPE_PREC_MIXED = 5
};

/* bank waveform element type */
enum { DOTPE_C128 = 0, DOTPE_C64 = 1 };

/* event flags */
#define DOTPE_FLAG_STORE_LNL 0x1   /* keep ln Lbar_ie and max_o ln L^ML_ie for dotpe_lnl_blocks */
#define DOTPE_FLAG_GEMM_ONLY 0x2   /* diagnostics: skip the marginalisation epilogue (result not valid) */
/* failure-path test: the tensor-core kernel's producer never signals its first
 * stage, so the consumer's bounded wait (0.25 s) runs out; the event ends FAILED
 * with DOTPE_E_TIMEOUT and the context stays usable.  Precisions other than FP32. */
#define DOTPE_FLAG_TEST_STALL 0x100

/* event states */
enum { DOTPE_STATE_QUEUED = 0, DOTPE_STATE_RUNNING = 1, DOTPE_STATE_DONE = 2, DOTPE_STATE_FAILED = 3 };

/* what dotpe_lnl_blocks returns */
enum {
  DOTPE_LNL_MARG = 0,   /* ln Lbar_ie = ln (1/N_phi) sum_o Lbar_ieo (Eq. lnl_dist_marginalized) */
  DOTPE_LNL_ML_MAX = 1, /* max_o ln L^ML_ieo (Eq. bestfit_lnl) */
  DOTPE_ROW_MARGINAL = 2, /* ln sum_{e,o} w_i w_e Lbar_ieo, one value per i (row e0..e1 ignored) */
  DOTPE_COL_MARGINAL = 3  /* ln sum_{i,o} w_i w_e Lbar_ieo, one value per e (rows ignored) */
};

/* ---- structures -------------------------------------------------------- */
typedef struct dotpe_ctx dotpe_ctx;

/* context flags */
/* time candidate tile forms (32-sample tiles; 64-sample tiles on one SM or on
 * CTA pairs) and L2 bands on the first event of each shape, keep the fastest */
#define DOTPE_CONFIG_AUTOTUNE 0x1
#define DOTPE_CONFIG_NO_GRAPHS 0x2 /* launch batches directly instead of as captured CUDA graphs */
/* Screening and GEMM-only launches of mode banks use 128 x 32-sample tiles
 * (two TMEM accumulator sets) instead of the default 128 x 64-sample tiles (one
 * set of N = 128 per mode, twice the MMA work per operand byte).  Results are
 * the same either way; with DOTPE_CONFIG_AUTOTUNE the tuner times both. */
#define DOTPE_CONFIG_NARROW_TILES 0x4
/* 64-sample tiles on one SM each instead of CTA pairs (two SMs sharing each
 * MMA, cta_group::2, each loading half of the extrinsic operand tile); the
 * autotuner then times no CTA pairs */
#define DOTPE_CONFIG_SINGLE_CTA_TILES 0x8

typedef struct dotpe_config {
  int device;                /* CUDA ordinal */
  uint64_t hbm_budget_bytes; /* device bytes the context may hold for banks + events; 0 = 90% of free */
  int n_slots;               /* launches (events or batches) that may run concurrently (0 = 4) */
  int flags;                 /* DOTPE_CONFIG_* */
  int max_batch;             /* continuous batching: up to this many queued events of one bank and
                                precision are admitted together as one batch (0 or 1: one at a time) */
} dotpe_config;

/* Intrinsic waveform bank on fixed bins (Sec. IV.C; h_{impb} stored on f_b only).
 * h: host or device, element type h_dtype, layout [n_int][n_modes][n_bins] complex.
 * f, w_quad: [n_bins] host or device doubles: bin frequencies (Hz) and quadrature
 * weights such that <a|b> = sum_d sum_b 4 w_quad[b] a b^* / S_d(f_b) (Eq. inner_product).
 * mode_m: host int [n_modes], azimuthal numbers, each in 1..4, distinct.
 * ln_w_int: [n_int] host or device, ln(pi/pi') of each sample (Eq. int_weights); NULL = 0.
 * pol: [n_int][n_modes][2] complex, host or device, or NULL: the polarisation
 *   factors K_{i m p} (p = +, x) of each row, h_{i m p} = K_{i m p} h_{i m}
 *   (App. B's h_impb, with the inclination an intrinsic parameter as in
 *   Sec. IV.A).  Only dotpe_preselect reads them; a bank without them cannot be
 *   pre-selected.  Kept on the device as FP32.
 * n_pol: 0 or 1 for the mode bank above; 2 for a polarisation-resolved bank
 *   (the general, precessing case of Sec. IV.A, Eqs. dh_ieo and hh_ieo with
 *   the polarisation index p): h is then [n_int][n_modes][2][n_bins] complex,
 *   h_{i m p b} with p = +, x, and each extrinsic sample carries real antenna
 *   patterns F_{e d p} (dotpe_event_desc.F) in place of R.  Every precision
 *   applies (the tensor-core kernels contract K = 4 n_bins, padded); its events
 *   are not batched with one another (dotpe_batch_submit in a precision other
 *   than DOTPE_PREC_FP32 returns DOTPE_E_UNSUPPORTED); relative binning takes
 *   weights per (mode, polarisation) component; dotpe_preselect takes it
 *   (the bank's own h_imp; pol is not needed) without relative binning. */
typedef struct dotpe_bank_desc {
  int64_t n_int;
  int n_modes;
  const int *mode_m;
  int n_bins;
  const double *f;
  const double *w_quad;
  const void *h;
  int h_dtype;
  const double *ln_w_int;
  const double *pol;
  int n_pol;
} dotpe_bank_desc;

/* One event: data, PSD, extrinsic samples (Sec. IV.B-E).
 * Rows [i0, i1) of the bank are used (N_int = i1 - i0).
 * psd [n_det][n_bins] (double), data [n_det][n_bins] (complex): host or device.
 * t [n_ext][n_det] (double, s): arrival time at each detector (Eq. t_at_detector).
 * R [n_ext][n_det][n_modes] (complex): response of mode m at detector d, i.e.
 *   the factor that multiplies h_m(f) T_d(f) Phi_m in Eq. h_k (polarisation sum folded in).
 * ln_w_ext [n_ext]: ln w_e (Sec. IV.E); NULL = 0.
 * u_min = d_L^0 / d_max of the distance prior pi(d_L) ~ d_L^2 on (0, d_max].
 * cut_delta > 0 enables the coherent-ML selection of Eq. coherent_ML_selection
 *   (phases with ln L^ML < max - cut_delta are not marginalised); <= 0 disables it.
 * stream: cudaStream_t the event's work is ordered after (NULL: none).
 * block_rows: 0 processes the slice in one pass; otherwise a positive multiple
 *   of 128: the slice streams through the kernels in blocks of that many bank
 *   rows (the event's device scratch then scales with block_rows, not with the
 *   slice), and each block's log-sum-exp partials, marginals and best ln L^ML
 *   are merged into FP64 accumulators in block order.  The result does not
 *   depend on block_rows beyond FP64 rounding, except where a maximum known
 *   block by block decides what is kept: the ML cut's superset, and in MIXED
 *   precision which tiles far below the maximum are refined.
 * rb_dh [n_det][J][n_bins], rb_hh [n_det][J][J][n_bins]
 *   (complex, host or device; both or neither; J = n_modes, or 2 n_modes
 *   (mode, polarisation) components j = 2m + p for a polarisation-resolved
 *   bank): relative-binning weights
 *   (App. A, from dotpe_rb_weights) replacing the plain quadrature: the data
 *   weight of component j becomes conj(W^{<d|h>}_{d j b}) and <h_j|h_j'>_d uses
 *   W^{<h|h>}_{d j j' b}.  psd and data are then not read (may be NULL); the
 *   cross-term cache is keyed by the <h|h> weights; the mixed-precision
 *   screening margin takes max_j sum_{d,b} |W^{<d|h>}_{d j b}|^2 / W^{<h|h>}_{d j j b}
 *   in place of <d|d>.
 * F [n_ext][n_det][2] (double, host or device): antenna patterns F_{e d p}
 *   (p = +, x) of each sample, read for a polarisation-resolved bank (n_pol = 2),
 *   which then ignores R (may be NULL).  A mode bank ignores F (may be NULL).
 * Without relative binning n_det * n_bins <= 58,112 (the <h|h> quadrature
 *   weights of all detectors are staged in 227 KB of shared memory); larger
 *   events return DOTPE_E_UNSUPPORTED. */
typedef struct dotpe_event_desc {
  uint64_t bank_id;
  int64_t i0, i1;
  int n_det;
  const double *psd;
  const double *data;
  int64_t n_ext;
  const double *t;
  const double *R;
  const double *ln_w_ext;
  int n_phi;
  double u_min;
  double cut_delta;
  int precision;
  int flags;
  void *stream;
  int64_t block_rows;
  const double *rb_dh;
  const double *rb_hh;
  const double *F;
} dotpe_event_desc;

typedef struct dotpe_event_stats {
  int64_t t_submit_ns, t_admit_ns, t_done_ns; /* host steady clock; 0 if not reached */
  int64_t n_pairs;                            /* N_int * N_ext */
  int64_t footprint_bytes;                    /* device bytes held while running */
  float device_ms;                            /* GPU time from first to last kernel */
  float prep_ms;                              /* data weights, extrinsic operand, cross terms */
  float fused_ms;                             /* fused GEMM + marginalisation kernel(s) */
  float refine_ms;                            /* MIXED: selection + refinement part of fused_ms; else -1 */
  int precision;
  int state;
} dotpe_event_stats;

/* Eq. Z_sum with w_o = 1; Eqs. posterior_element, int_ess, ext_ess; Eq. bestfit_lnl. */
typedef struct dotpe_evidence_out {
  double ln_z;              /* ln Z = ln[(1/(N_i N_e N_phi)) sum_ieo w_i w_e Lbar_ieo] */
  double n_eff, n_eff_int, n_eff_ext;
  double max_lnl_ml;        /* max over (i,e,o) of ln L^ML */
  int64_t arg_i, arg_e, arg_o; /* its location (i in bank numbering); lowest (i,e,o) on ties */
  int64_t n_marginalised;   /* (i,e,o) for which Lbar was evaluated */
  int64_t n_pairs;
  double lnl_ml_threshold;  /* the cut applied (running maximum - cut_delta), -inf when off */
  int32_t device_status;    /* 0, or a DOTPE_E_* raised inside a kernel */
  int32_t n_refined_tiles;  /* MIXED: tiles recomputed in split precision; else -1 */
  /* MIXED: pairs that passed the screening pass's first bound (64-sample tiles:
   * sum_m |Z_m| against the <h|h> lower bound; 32-sample tiles: the pairs taken
   * for evaluation), and pairs whose ln L^ML the screen evaluated over the phase
   * grid; else -1.  Diagnostics of the screen's selectivity, not of the result. */
  int64_t n_screen_candidates, n_screen_evaluated;
} dotpe_evidence_out;

/* Incoherent single-detector pre-selection of bank rows (Sec. IV.D, App. B).
 * Each detector k on its own, over a grid of arrival times t_{kt} and the
 * orbital-phase grid phi_o = 2 pi o / n_phi, with the two polarisation
 * amplitudes free (App. B: for one detector, sky position, distance and
 * polarisation angle reduce to them):
 *   <d|h>_{i k o t p} = Re sum_{m,b} 4 w_b d_k^*(f_b) / S_k(f_b) K_{imp} h_{im}(f_b)
 *                        e^{-2 pi i f_b t_{kt}} e^{i m phi_o}               (Eq. dh_itop)
 *   <h|h>_{i k o p p'} = Re sum_{m,m',b} 4 w_b / S_k(f_b) K_{imp} h_{im} K^*_{im'p'} h^*_{im'}
 *                        e^{i (m - m') phi_o}
 *   ln L^ML_{i k o t} = dh^T [hh]^+ dh / 2                                   (Eqs. x_ML, single_det_ML)
 *   ln L^inco.ML_i = sum_k max_{o,t} ln L^ML_{i k o t}, and row i is kept when
 *   ln L^inco.ML_i >= max_j ln L^inco.ML_j - delta                          (Sec. IV.D, delta = 20 there)
 * [hh]^+ is the inverse when det > 1e-3 hh_{++} hh_{xx}, else the rank-one
 * pseudo-inverse hh / (hh_{++} + hh_{xx})^2 (a row seen edge-on has hx = 0).
 * The phase factor's sign differs from App. B's e^{-i m phi}; the grid is
 * closed under phi -> -phi, so the maxima are the same.
 * The <d|h> components are one tensor-core GEMM per mode against the bank's
 * operand planes (precision FP16, FP16X3, BF16 or BF16X3); the rest is FP32,
 * the detector sum and the selection FP64.  A polarisation-resolved bank
 * (n_pol = 2) uses its own h_{imp} in place of K_{imp} h_{im} (App. B's
 * general form; pol is not needed): the tensor-core precisions as above, or
 * DOTPE_PREC_FP32 on the CUDA cores; with relative binning it runs in FP32
 * only (other precisions return DOTPE_E_UNSUPPORTED), with the component
 * weights rb_dh [n_det][2M][n_bins], rb_hh [n_det][2M][2M][n_bins] (j = 2m + p)
 * and one time-grid operand per component.
 * Rows [i0, i1) of the bank.
 * psd [n_det][n_bins] (double) and data [n_det][n_bins] (complex): host or
 * device, as for events.  t_grid [n_det][n_t] (double, s; host or device):
 * the arrival times at each detector.  1 <= n_t <= 4096, 1 <= n_phi <= 32,
 * delta >= 0.  rb_dh / rb_hh as in dotpe_event_desc (relative binning, App. A;
 * the weights do not depend on the polarisation for a reference h0_{mp} =
 * K_{mp} h0_m, so for a mode bank the per-mode weights serve both
 * polarisations); the time grid operand is then one per mode (per component
 * for a polarisation-resolved bank).  Synchronous: returns when every output
 * is written. */
typedef struct dotpe_presel_desc {
  uint64_t bank_id;
  int64_t i0, i1;
  int n_det;
  const double *psd;
  const double *data;
  int n_t;
  const double *t_grid;
  int n_phi;
  double delta;
  int precision;
  int flags; /* 0 */
  const double *rb_dh;
  const double *rb_hh;
} dotpe_presel_desc;

typedef struct dotpe_presel_out {
  double max_lnl_inco; /* max_i ln L^inco.ML_i */
  double threshold;    /* max_lnl_inco - delta */
  int64_t arg_i;       /* lowest row (slice-relative) attaining the maximum */
  int64_t n_selected;  /* N_int' of Sec. IV.D */
  float kernel_ms;     /* device time of the GEMM + single-detector ML kernel */
  float device_ms;     /* device time of the whole call (preparation to selection) */
  int32_t device_status; /* 0, or a DOTPE_E_* raised inside a kernel */
} dotpe_presel_out;

/* Relative-binning weights (App. A, Eqs. dh_weights, hh_weights) of one
 * event for a bank stored on coarse nodes of a fine frequency grid:
 *   W^{<d|h>}_{d m b}    = <d_d | h0_dm s_b> / h0_dm^*(f_b)
 *   W^{<h|h>}_{d m m' b} = <h0_dm | h0_dm' s_b> / (h0_dm(f_b) h0_dm'^*(f_b))
 * with <a|b> = sum_n 4 df_fine[n] a(f_n) b^*(f_n) / S_d(f_n) on the fine grid,
 * h0_dm(f) = h0_m(f) e^{-2 pi i f t0_d} (the reference waveform's modes
 * arriving at detector d at t0_d), s_b the piecewise-linear hat function of
 * node b (1 at f_b = f_fine[nodes[b]], 0 at the neighbouring nodes; the fine
 * points outside [f_0, f_{B-1}] do not enter).  Then <d|h_m>_d is
 * approximated by sum_b W^{<d|h>}_{d m b} h_m^*(f_b) and <h_m|h_m'>_d by
 * sum_b W^{<h|h>}_{d m m' b} h_m(f_b) h_m'^*(f_b) (Eqs. d_h, h_h), which
 * dotpe_event_desc.rb_dh / rb_hh and dotpe_presel_desc.rb_dh / rb_hh take.
 * The bank's bins must be the node frequencies.  f_fine [n_fine] (increasing),
 * df_fine [n_fine] (quadrature weights), psd [n_det][n_fine],
 * data [n_det][n_fine] complex, h0 [n_modes][n_fine] complex, t0 [n_det]
 * (may be NULL: 0), nodes [n_bins] (strictly increasing indices into
 * f_fine): host or device.  Computed on the device in FP64.
 * n_modes counts components, 1..8: the modes of a mode bank, or, for a
 * polarisation-resolved bank, its (mode, polarisation) pairs j = 2m + p with
 * h0 [2 M][n_fine] the reference's h0_{mp} (the weights then carry the
 * polarisation index, W_{d m p b} and W_{d m m' p p' b}, as App. A writes them). */
typedef struct dotpe_rb_desc {
  int n_det, n_modes;
  int64_t n_fine;
  const double *f_fine;
  const double *df_fine;
  const double *psd;
  const double *data;
  const double *h0;
  const double *t0;
  int n_bins;
  const int64_t *nodes;
} dotpe_rb_desc;

/* ---- context ----------------------------------------------------------- */
/* Creates a context on cfg->device (cfg may be NULL: defaults) and its
 * streams.  The distance-marginal lookup table of Eq. lnl_dist_marginalized
 * lives in static device memory (3.2 MB per GPU that loads the library, held
 * until the process exits); the first context created in a CUDA context of
 * the device builds it (about 0.1 s of FP64 work), later ones share it.
 * Errors: E_INVALID (bad device), E_DEVICE, E_NOMEM. */
int dotpe_create(const dotpe_config *cfg, dotpe_ctx **out);

/* Waits for outstanding work, frees every bank/event and the context. */
int dotpe_destroy(dotpe_ctx *ctx);

const char *dotpe_strerror(int status);
const char *dotpe_last_error_message(void);
int dotpe_version(void);

/* Number of SMs and the name of the device the context runs on. */
int dotpe_device_info(dotpe_ctx *ctx, int *n_sms, char *name, int name_len);

/* ---- bank -------------------------------------------------------------- */
/* Copies the bank to the device (synchronously) and prepares the operand
 * planes of every precision: FP32 master, bf16 hi/lo, fp16; rows padded to
 * a multiple of 64 frequency-pairs.  The caller keeps its buffers.
 * Errors: E_INVALID (shape, mode numbers, non-finite values), E_NOMEM
 * (beyond the HBM budget), E_DEVICE. */
int dotpe_bank_load(dotpe_ctx *ctx, const dotpe_bank_desc *desc, uint64_t *bank_id);

/* Frees a bank.  E_INVALID if an unreleased event still uses it. */
/* A new bank holding rows[0..n) of bank bank_id, in that order (Sec. IV.D:
 * the coherent stage runs on the rows the pre-selection keeps; its
 * `selected` output is a valid row list).  The rows' waveforms are copied on
 * the device as the bank holds them (FP32 master and both operand formats,
 * same scale), with their ln w_int and polarisation factors, so an event over
 * the new bank gives, pair by pair, the values of the parent bank's rows.
 * rows: int64 [n], host or device, each in [0, n_int) (repeats allowed).
 * Errors: E_INVALID (null argument, n < 1, a row out of range), E_NOT_FOUND,
 * E_NOMEM (beyond the HBM budget), E_DEVICE. */
int dotpe_bank_subset(dotpe_ctx *ctx, uint64_t bank_id, const int64_t *rows, int64_t n, uint64_t *new_bank_id);

/* Checkpoint / resume of a resident bank: dotpe_bank_save writes it to the
 * file `path` (a header with the shapes, mode numbers and operand scale, then
 * f, w_quad, ln w_int, the FP32 master rows and the polarisation factors, and
 * an FNV-1a 64 checksum of them); dotpe_bank_open loads such a file as a new
 * bank whose operands equal the saved bank's (the bf16/fp16 planes are
 * rebuilt at the saved scale), so its events give the same values.  The file
 * is in the host's byte order.  Errors: E_INVALID (null argument, unreadable
 * or unwritable file, wrong magic or version, inconsistent header, truncated
 * payload, checksum mismatch), E_NOT_FOUND, E_NOMEM, E_DEVICE. */
int dotpe_bank_save(dotpe_ctx *ctx, uint64_t bank_id, const char *path);
int dotpe_bank_open(dotpe_ctx *ctx, const char *path, uint64_t *bank_id);
int dotpe_bank_release(dotpe_ctx *ctx, uint64_t bank_id);

/* ---- events ------------------------------------------------------------ */
/* Queues one event and returns at once (inputs are copied before return).
 * The event is admitted as soon as its device footprint fits the free part of
 * the HBM budget and a slot is free; admitted events run concurrently on the
 * device.  Errors: E_INVALID, E_NOT_FOUND (bank), E_ADMISSION (footprint larger
 * than the whole budget), E_NOMEM. */
int dotpe_event_submit(dotpe_ctx *ctx, const dotpe_event_desc *desc, uint64_t *event_id);

/* Queues n events that share one bank and one precision as one batch: they are
 * admitted together (the sum of their footprints) and run as one launch
 * sequence on one slot: every event's preparation, then one persistent fused
 * tcgen05 launch per 64 events whose work items are the events' tiles one
 * event after the other (mixed precision: one screening launch, one selection
 * over the batch, one refinement launch), then every event's reduction.  The
 * sequence is captured as a CUDA graph (unless DOTPE_CONFIG_NO_GRAPHS) whose
 * executable is kept per slot and updated in place for the next batch.  Each
 * event's results are those it gets when submitted alone (same tiles, same
 * per-event reductions).  descs[k].block_rows must be 0.  event_ids: [n] out.
 * The paper has no counterpart (it evaluates one event at a time, Sec. IV).
 * Errors: as dotpe_event_submit for any event (then none is queued);
 * E_INVALID (banks or precisions differ, block_rows != 0); E_ADMISSION (the
 * batch can never fit the budget). */
int dotpe_batch_submit(dotpe_ctx *ctx, int n, const dotpe_event_desc *descs, uint64_t *event_ids);

/* Non-blocking state query; also admits queued events whose memory now fits.
 * stats may be NULL.  Errors: E_NOT_FOUND. */
int dotpe_event_poll(dotpe_ctx *ctx, uint64_t event_id, int *state, dotpe_event_stats *stats);

/* Blocks until the event is DONE or FAILED, at most timeout_s seconds
 * (<= 0: no limit).  Errors: E_TIMEOUT, E_NOT_FOUND, E_DEVICE. */
int dotpe_event_wait(dotpe_ctx *ctx, uint64_t event_id, double timeout_s);

/* Makes `stream` (a cudaStream_t) wait, on the device, for the event's
 * completion.  Returns once the wait is enqueued; while the event is still
 * queued (not yet admitted) the call blocks on the host until it is.
 * Errors: E_NOT_FOUND, E_DEVICE. */
int dotpe_event_stream_wait(dotpe_ctx *ctx, uint64_t event_id, void *stream);

/* Evidence, effective sample sizes and the ML point of a finished event.
 * Errors: E_NOT_READY, E_NOT_FOUND, E_DEVICE (device_status set). */
int dotpe_evidence(dotpe_ctx *ctx, uint64_t event_id, dotpe_evidence_out *out);

/* Copies a block of per-pair or marginal results into out (host or device),
 * row-major with leading dimension ld (floats); i and e are relative to the
 * event's slice.  LNL_MARG / LNL_ML_MAX come from the stored values when the
 * event ran with DOTPE_FLAG_STORE_LNL; otherwise the block is recomputed
 * synchronously from the event's inputs (kept until dotpe_event_release), in
 * the event's arithmetic (split fp16 for MIXED), with the ML cut fixed at the
 * event's final threshold (lnl_ml_threshold), on memory outside the budget
 * for the duration of the call.
 * ROW_MARGINAL writes out[k] for i = i0+k; COL_MARGINAL out[k] for e = e0+k.
 * Errors: E_NOT_READY, E_NOT_FOUND, E_INVALID (range), E_NOMEM, E_DEVICE. */
int dotpe_lnl_blocks(dotpe_ctx *ctx, uint64_t event_id, int64_t i0, int64_t i1, int64_t e0,
                     int64_t e1, int what, float *out, int64_t ld);

/* Posterior samples of a finished event by resampling (Sec. III: the weights
 * p_ieo = w_i w_e w_o Lbar_ieo of Eq. posterior_element, w_o = 1) with a
 * distance drawn per sample from the summand of the distance marginal
 * (App. C).  The caller supplies the random numbers: uniforms [n][4] in
 * [0, 1) (host or device).  Per sample: u1 picks the bank row i (weights
 * sum_{e,o} p_ieo, the event's FP64 row marginals), u2 the extrinsic sample e
 * (weights w_e Lbar_ie of the stored row), u3 the phase o (weights Lbar_ieo
 * of the phases that pass the event's ML cut, the pair recomputed in FP64 from
 * the event's inputs), u4 the distance: d_L / d_L^0 = 1/u with u on
 * [u_min, inf) of density proportional to u^-4 exp(dh_o u - hh_o u^2 / 2).
 * Each draw takes the smallest index whose cumulative weight exceeds u times
 * the total.  The paper draws N_s = N_eff / 2 samples (Sec. V.B).  Outputs
 * (host or device, each may be NULL): i_out [n] (slice-relative), e_out [n],
 * o_out [n], dist_out [n].  The event must be DONE and must have run with
 * DOTPE_FLAG_STORE_LNL.  Errors: E_NOT_FOUND, E_NOT_READY, E_INVALID (no
 * stored values, n not in 1..2^24, no pair of positive weight), E_NOMEM,
 * E_DEVICE. */
int dotpe_posterior_samples(dotpe_ctx *ctx, uint64_t event_id, int64_t n, const double *uniforms,
                            int64_t *i_out, int64_t *e_out, int32_t *o_out, double *dist_out);

/* Frees an event's device state.  A RUNNING event is waited for first; a
 * QUEUED event (not yet admitted to a slot) is cancelled: it never runs, and
 * the events queued behind it are admitted in order.  The id is invalid
 * afterwards (E_NOT_FOUND).  Errors: E_NOT_FOUND. */
int dotpe_event_release(dotpe_ctx *ctx, uint64_t event_id);

/* ---- relative binning -------------------------------------------------- */
/* Computes the weights of dotpe_rb_desc into w_dh [n_det][n_modes][n_bins]
 * and w_hh [n_det][n_modes][n_modes][n_bins] (complex, host or device, owned
 * by the caller).  Synchronous; temporary device memory outside the HBM
 * budget for the call.  Errors: E_INVALID (shapes, nodes not strictly
 * increasing or out of range, non-finite or non-positive PSD, a reference
 * mode that vanishes at a node), E_NOMEM, E_DEVICE. */
int dotpe_rb_weights(dotpe_ctx *ctx, const dotpe_rb_desc *desc, double *w_dh, double *w_hh);

/* ---- pre-selection ----------------------------------------------------- */
/* Runs the pre-selection of dotpe_presel_desc on the bank's rows [i0, i1)
 * (N = i1 - i0) and writes, into host or device buffers the caller owns
 * (each may be NULL):
 *   lnl_ml   [N][n_det] float   max_{o,t} ln L^ML_{i k o t}
 *   arg_ot   [N][n_det][2] int  its (o, t); lowest t, then lowest o, on ties
 *   lnl_inco [N] double         ln L^inco.ML_i
 *   selected [N] int64          the kept rows (slice-relative) in increasing
 *                               order; the first out->n_selected are valid
 * The <h|h>_k mode overlaps come from the bank's cross-term cache for this
 * PSD when an event has filled it, else are computed for the slice.
 * Temporary device memory (about N (4 n_det + 2) x 8 bytes plus the packed
 * time-grid operand) is taken outside the HBM budget for the call.
 * Errors: E_INVALID (shape, range, precision, a bank without pol, non-finite
 * input), E_NOT_FOUND (bank), E_NOMEM, E_TIMEOUT (a device wait ran out),
 * E_DEVICE. */
int dotpe_preselect(dotpe_ctx *ctx, const dotpe_presel_desc *desc, float *lnl_ml, int32_t *arg_ot,
                    double *lnl_inco, int64_t *selected, dotpe_presel_out *out);

/* ---- bank-sharded events ------------------------------------------------ */
/* One event whose bank slice is split by rows into shards (e.g. one shard per
 * GPU, each shard an event of its own over the same extrinsic samples): the
 * paper's sums over i are plain sums (Eq. Z_sum; Eqs. posterior_element,
 * int_ess, ext_ess), so the shards combine exactly, in FP64 on the host:
 *   ln S1 = LSE_r [ln Z_r + ln(N_i,r N_e N_phi)],  ln Z = ln S1 - ln(N_i N_e N_phi),
 *   sum p^2 and sum_i P_i^2 add over shards (recovered from each shard's N_eff
 *   and N_eff,int), the per-sample marginals P_e add over shards (then
 *   N_eff,ext = S1^2 / sum_e P_e^2), the maximum ln L^ML is the largest (lowest
 *   (i, e, o) on ties).  Calls no CUDA function. */
typedef struct dotpe_shard {
  dotpe_evidence_out ev;   /* the shard's evidence (dotpe_evidence); arg_i in bank numbering */
  int64_t n_int;           /* rows of the shard's slice */
  const double *ln_p_ext;  /* [n_ext] host: the shard's per-sample marginals, ln sum_{i,o} w_i w_e Lbar_ieo
                              (dotpe_lnl_blocks with DOTPE_COL_MARGINAL, widened to double) */
} dotpe_shard;
/* shards: n_shards >= 1 records over the same n_ext samples and n_phi phases.
 * out: the event's evidence (n_marginalised and n_pairs summed; lnl_ml_threshold
 * the largest of the shards'; device_status the first nonzero; n_refined_tiles
 * summed, -1 if any shard has -1).  ln_p_ext_out: [n_ext] host or NULL, the
 * event's per-sample marginals.  Errors: E_INVALID (null pointers, n_shards <
 * 1, n_ext < 1, n_int < 1, n_phi < 1). */
int dotpe_evidence_merge(int n_shards, const dotpe_shard *shards, int64_t n_ext, int n_phi,
                         dotpe_evidence_out *out, double *ln_p_ext_out);

/* ---- diagnostics ------------------------------------------------------- */
/* Evaluates the device distance marginal ln Lbar(dh, hh) (Eq.
 * lnl_dist_marginalized with pi(d_L) ~ d_L^2, u_min = d0/d_max) for n inputs.
 * dh, hh, out: host or device float arrays of length n.  Runs the same device
 * function as the fused epilogue. */
int dotpe_dist_marg_eval(dotpe_ctx *ctx, int64_t n, const float *dh, const float *hh, float u_min,
                         float *out);

/* Allocation-free variant of dotpe_dist_marg_eval (the paper has no
 * counterpart; this is a library service).  Some callers cannot allocate
 * device memory at the point where they call: hosts that hand the whole
 * device to their own allocator (a framework's caching allocator that has
 * reserved all free memory, so a cudaMalloc of ours would fail or fragment
 * it), and latency-bound loops that must not pay for cudaMalloc/cudaFree and
 * the synchronisation cudaFree implies.  This entry point calls no
 * cudaMalloc, cudaFree or other allocating routine.  Its scratch for the
 * inputs and the output is a static device array of 3 x 2^20 floats (12 MiB)
 * that every GPU loading the library holds until the process exits; the
 * array's device address is looked up with cudaGetSymbolAddress on the
 * first call on each device (and again after the device's context has been
 * replaced, e.g. by cudaDeviceReset), so make that first call before any
 * stream capture.  n must not exceed 2^20 (1,048,576): larger n is rejected with
 * DOTPE_E_INVALID and a message.  dh, hh, out: host or device float arrays
 * of length n, as for dotpe_dist_marg_eval.  All calls share the one scratch
 * array and are serialised on the context's stream; calls that overlap on
 * the GPU (e.g. from several contexts on one device) race on it.  The call
 * returns after the result is in `out`.  Errors: E_INVALID, E_DEVICE. */
int dotpe_dist_marg_eval_noalloc(dotpe_ctx *ctx, int64_t n, const float *dh, const float *hh, float u_min,
                                 float *out);

#ifdef __cplusplus
}
#endif
#endif /* DOTPE_H */
