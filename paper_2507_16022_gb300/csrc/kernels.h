// Host-side launchers of the dotpe kernels (internal).
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace dotpe {

// fp16 operands are scaled to magnitudes up to 2^14 instead of 1: the five
// exponent bits then keep hi normal down to ~4e-9 of the largest element and lo
// (~2^-11 hi) normal down to ~8e-6 of it, so the split keeps ~2^-22 relative
// accuracy over the data's dynamic range (products and K-sums stay far inside FP32).
constexpr float FP16_OPERAND_SCALE = 16384.0f;

struct PrepArgs {
  int D, B, M, Kpad;
  int64_t E;
  // inputs (device)
  const double *f, *w, *psd;
  const double2 *data;
  const double *t;
  const double2 *R;
  // outputs (device)
  float2 *c;
  float *omega, *fh, *fl, *th, *tl;
  float2 *Rf;
  float *qx;
  float2 *G32;     // [M][E][B]
  float *gmax;     // 1 float, zeroed
  void *gpack;     // packed operand planes
  int pack_kind;   // 0 fp32, 1 bf16, 2 fp16
  int pack_planes; // 1 or 2 (hi, lo)
  float *gscale;   // 1 float out
  float *sqrt_dd;  // 1 float out: sqrt<d|d> (Eq. inner_product, FP64 sum)
  int *status;
  // relative binning (App. A), both or neither: W^{<d|h>} [D][J][B], W^{<h|h>} [D][J][J][B]
  // over the J = M n_pol (mode, polarisation) components
  const double2 *rb_dh, *rb_hh;
  // polarisation-resolved bank (n_pol = 2): real antenna patterns F [E][D][2] replace R;
  // G32 is then [M][2][E][B] and the packed rows carry two polarisation blocks along K
  int n_pol;
  const double *F;
};

void launch_prep(const PrepArgs &a, cudaStream_t st);
// rb_hh non-null: relative-binning mode-pair weights instead of omega
void launch_cross_terms(int64_t n_rows, int64_t row0, int64_t I_bank, int M, int D, int B, int Kpad,
                        const float *master, const float *omega, const double2 *rb_hh, float *mx, int n_sms,
                        cudaStream_t st);
void launch_bank_to_master(int64_t rows, int64_t row0, int64_t I_bank, int M, int B, int Kpad, int NP,
                           const void *src, int dtype, float *master, float *amax, int *status, cudaStream_t st);
// polarisation-resolved bank: row records of REC_P floats per detector (kernels_prep.cu);
// rb_hh non-null: relative-binning weights per component pair [D][2M][2M][B] instead of omega
void launch_cross_terms_pol(int64_t n_rows, int64_t row0, int64_t I_bank, int M, int D, int B, int Kpad,
                            const int *mode_m, const float *master, const float *omega, const double2 *rb_hh,
                            float *mx, int n_sms, cudaStream_t st);
// dst[o][r][:] = src[o][rows[r]][:], rows of row_words 32-bit words (device rows[n], in range)
void launch_gather_rows(int64_t outer, int64_t src_rows, int64_t n, int64_t row_words, const void *src,
                        const int64_t *rows, void *dst, cudaStream_t st);
void launch_master_to_planes(int64_t n, const float *master, const float *amax, __nv_bfloat16 *bf /*[2][n]*/,
                             __half *hf /*[2][n]*/, float *scale_out, cudaStream_t st);
// The device's distance-marginal table (static device memory), built on `st`
// on first use in the current CUDA context of `device` (which must be current);
// later calls return the same address.  DOTPE_OK, or an error code with `msg`.
int shared_dm_table(int device, cudaStream_t st, float4 **tab, char *msg, size_t msg_len);
void launch_dist_marg_eval(int64_t n, const float *dh, const float *hh, float u_min, const float4 *tab, float *out,
                           cudaStream_t st);
constexpr int64_t DM_NOALLOC_MAX = 1 << 20;  // evaluations per allocation-free call
int dist_marg_eval_noalloc(int device, int64_t n, const float *dh, const float *hh, float u_min, const float4 *tab,
                           float *out, cudaStream_t st, char *msg, size_t msg_len);

// Fused <d|h> GEMM + marginalisation epilogue, FP32 SIMT (plain path).
struct SimtArgs {
  const float *A;   // FP32 master [M][I_bank][Kpad]
  const float *Bm;  // FP32 packed G [M][2E][Kpad]
  int64_t I_bank;
  int Kpad, K;      // K = 2B (multiple-of-8 not required)
};
constexpr int SIMT_TI = 64, SIMT_TE = 32;
void launch_simt(const SimtArgs &g, const EpiParams &P, cudaStream_t st);

// Fused tcgen05 kernel over a batch of events sharing one bank.
constexpr int TC_TI = 128, TC_TE = 32;
constexpr int TC_MAXB = 64;  // events per batched launch (kernel-parameter space)
struct TcEvent {             // one event of a launch (without its tensor map)
  EpiParams P;
  int n_itile, n_etile, band;      // tiles of the event (block) and its L2 band width
  int a_row0;                      // first bank row of the event's slice (block)
  int b_plane_rows, b_mode_rows;   // rows of one operand plane / one mode in mapB
};
struct TcWork : TcEvent {    // host-side record: the event and its maps
  CUtensorMap mapB;          // packed extrinsic operand planes [planes][M][2E][Kpad], 64-row boxes
  CUtensorMap mapB64;        // the same planes in 128-row boxes (64-sample tiles); zero if not encoded
};
template <int NB>
struct TcBatch {
  CUtensorMap mapB[NB];
  TcEvent w[NB];
  int begin[NB + 1];     // grid mode: event k owns work items [begin[k], begin[k+1])
  int n;                 // events
  const int2 *glist;     // list mode (device): work item -> (event, linear tile it * n_etile + et)
  const int *glist_n;    // its length (device)
  const int *gate;       // optional [n] per event: items of event k run only if gate[k] == gate_want
  int gate_want;
};
struct TcCommon {
  int kb;                          // k-blocks of 64 per mode (Kpad / 64)
  int a_plane_rows, a_mode_rows;   // bank rows of one plane / one mode in mapA
  int n_modes;
};
struct TcLaunch {
  CUtensorMap mapA;  // bank operand planes [planes][M][I][Kpad]
  TcCommon C;
  bool bf16, split, consec;
  bool pol;          // polarisation-resolved bank (row records in registers, n_det <= POL_TC_MAXD)
  bool sep;          // split: hi*lo + lo*hi in their own accumulator (see kernel_tc.cuh)
  int tev;           // extrinsic samples per work tile: 32, or 64 (single-pass mode banks, grid order)
  bool pair;         // 64-sample tiles of one event: CTA pairs (cta_group::2, M = 256)
  const int *gate;   // optional device words per event: event k's items run only if gate[k] == gate_want
  int gate_want;
  int n_sms;
};
// A refinement whose screened maximum ln L^ML exceeds this uses the separate
// low-order accumulator: below it, one shared FP32 accumulator keeps the
// tensor-core truncation floor (~7e-6 ln L^ML at Kpad = 1024) under 1e-3.  The
// floor grows with the accumulation chain, so longer K lowers the threshold in
// proportion (SEP_ML 1024 / Kpad for Kpad > 1024).
constexpr float SEP_ML = 140.0f;
// n <= TC_MAXB works; glist/glist_n non-null for list mode.  Returns a cudaError_t.
int launch_tc(const TcLaunch &L, const TcWork *works, int n, const int2 *glist, const int *glist_n, cudaStream_t st);
// extrinsic tiles per L2 band: the band's operand planes fill about l2_band_bytes
int tc_band(double l2_band_bytes, int kb, int n_modes, bool split, int n_etile);

// K4 on the tensor cores (kernel_hh.cu): a lower bound of <h|h> at every phase
// for every pair of a bank block and an event, C_0 - 2 sum_delta |C_delta| less
// 2^-8 C_0, as bf16 rounded down [rows][hb_ld(E)]; the screening pass reads it.
struct HbDelta {
  int pdelta[NPAIR];  // m_a - m_b of mode pair p (a > b), 1..3; 0 for pairs beyond the modes
};
struct HbArgs {
  int64_t n_rows;
  int n_itile, n_etile;           // 128-row tiles, 32-sample tiles
  int a_plane_rows, b_plane_rows; // rows of one bf16 plane of the row records / sample matrix
  int n_kstep;                    // 16-entry K steps that hold record entries (one per detector)
  __nv_bfloat16 *out;             // [n_rows][ld]
  int64_t ld;
  int *status;
};
int64_t hb_ld(int64_t E);
// device scratch of launch_hh_bound (record planes and the bound itself)
size_t hb_scratch_bytes(int64_t rows, int64_t E);
// mx [rows][D][REC] row records of the block, qx [E][D][REC] column records; *out set to
// the bound inside `scratch`.  Returns 0, or < 0 if a launch or a tensor map failed.
int launch_hh_bound(int64_t rows, int64_t E, int D, const HbDelta &dl, const float *mx, const float *qx,
                    void *scratch, __nv_bfloat16 **out, int n_sms, int *status, cudaStream_t st);

// Refinement selection after a screening pass, over a batch of events: the
// tiles whose screened best ln L^ML can reach the cut, in banded tile order,
// written as (event, tile) work items.
struct SelectEvent {
  const float *tile_ml;    // [n_itile * n_etile] screened best ln L^ML per tile (-1: none evaluated)
  int n_itile, n_etile, band;
  const float *ml_screen;  // screened running maximum
  const float *sqrt_dd;    // sqrt<d|d>
  float window;            // tiles within window + 2 margins of the maximum are refined
  float margin_k;          // kappa*u of the screening precision
  float sep_ml;            // screened maxima above this take the separate low-order accumulator
  float *ml_refine;        // out: screened maximum - margin (a lower bound of the exact maximum)
  int *n_refined;          // out: the event's refined tiles
};
struct SelectBatch {
  SelectEvent ev[TC_MAXB];
  int begin[TC_MAXB + 1];  // event k's tiles are [begin[k], begin[k+1]) of the batch
  int n;
  int2 *list;              // out: (event, tile) items, event by event
  int *n_list;             // out: total
  int *counts;             // scratch: select_count_blocks(begin[n]) ints
  int *sep;                // out [n]: 1 where the event's screened maximum exceeds SEP_ML
};
int select_count_blocks(int n_tiles);
void launch_select(const SelectBatch &a, cudaStream_t st);

// Cross-tile FP64 reduction -> evidence, one bank block at a time.
struct ReduceOut {
  double ln_z, ln_s1, ln_s2, n_eff, n_eff_int, n_eff_ext;
  double max_ml;
  long long arg;
  long long n_marg;
  double threshold;
  int status;
  int n_refined;  // tiles refined in split precision (mixed), else -1
  long long n_cand, n_eval;  // screening statistics (mixed), else -1
};
// FP64 accumulators across bank blocks: (m, s) pairs with s = 0 meaning empty.
struct EvAcc {
  double s1_m, s1_s, s2_m, s2_s, pi_m, pi_s;  // ln S1, ln S2, ln sum_i P_i^2
  float best;                                 // best ln L^ML so far
  long long arg;                              // its packed (i, e, o), i relative to the slice
  long long n_marg;
};
struct ReduceArgs {
  int64_t n_int, n_ext;  // rows of this block, extrinsic samples
  int64_t row_offset;    // first row of the block within the slice
  int64_t n_int_total;   // rows of the slice
  int n_itile, n_etile, n_phi;
  int first;             // first block: accumulators start empty
  const float4 *tile_part;
  const float2 *row_part, *col_part;
  const float *tile_ml;
  const long long *tile_arg;
  const int *tile_npass;
  const float *ml_running;
  float cut_delta;
  double *ln_p_int;  // [n_int_total] out (slice)
  double *ln_p_ext;  // [n_ext] out (final kernel)
  EvAcc *acc;        // device
  double2 *acc_col;  // [n_ext] device
  void *scratch;     // reduce_scratch_bytes() of device memory
  const int *status;
  const int *n_refined;  // optional
  const unsigned long long *n_cand;  // optional: the screen's two counters
  ReduceOut *out;
};
void launch_reduce_block(const ReduceArgs &a, cudaStream_t st);
void launch_reduce_final(const ReduceArgs &a, cudaStream_t st);
size_t reduce_scratch_bytes();

// Incoherent single-detector pre-selection (Sec. IV.D, App. B): kernel_presel.cu.
constexpr int PS_TC = 64;       // (detector, time) columns per tile; time grids are padded to a multiple
constexpr int PS_TR = 64;       // bank rows per tile
constexpr int PS_MAXPHI = 32;   // phases per grid
constexpr float PS_RANK_TOL = 1e-3f;  // [hh]^+ is the rank-one limit when det <= PS_RANK_TOL hh_++ hh_xx
struct PreselPrepArgs {
  int D, B, M, Kpad, n_t, n_tpad;
  const double *f, *w, *psd;
  const double2 *data;
  const double *t_grid;  // [D][n_t]
  const double2 *rb_dh;  // relative binning (App. A) or null: then G is per weight component
  float2 *c;             // [D][M][B] data weights of each component (M: modes, or the 2 n_modes
                         // (mode, polarisation) components of a polarisation-resolved bank with rb_dh)
  float *omega, *fh, *fl;
  float2 *G32;           // [1 or M][D n_tpad][B] c_{kmb} e^{-2 pi i f_b t_{kt}} (0 on padding columns)
  float *gmax;           // 1 float, zeroed
  void *gpack;           // packed operand planes [planes][2 D n_tpad][Kpad]
  int pack_kind;         // 0 none (FP32 operand used as it is), 1 bf16, 2 fp16
  int pack_planes;       // 1 or 2 (hi, lo)
  float *gscale;         // 1 float out
  int *status;
};
void launch_presel_prep(const PreselPrepArgs &a, cudaStream_t st);
struct PreselParams {
  int n_rows;            // rows of the slice
  int a_row0;            // first bank row of the slice
  int n_det, n_t, n_tpad, n_phi, n_modes;
  int mode_m[MAXM];
  int pdelta[NPAIR];     // m_a - m_b of mode pair p (a > b), 1..3
  int slot[MAXM];        // epilogue mode slots: bank mode index (even m first, or by m mod 4 when quad)
  int n_even;            // modes with even m
  int quad;              // mode bank, n_phi % 4 == 0, one mode per class m mod 4: slot s holds class
                         // (0, 2, 1, 3)[s] and the phases are taken four at a time (phi + k pi / 2)
  unsigned slot_mask;    // slots that hold a mode (the others are empty)
  int n_itile, n_ctile;  // 64-row tiles, 64-column tiles
  int kb;                // k-blocks of 64 per mode
  int a_plane_rows, a_mode_rows, b_plane_rows;
  int b_mode_rows;       // per-mode time-grid operand (relative binning): rows of one mode, else 0
  const float2 *pol;     // [n_rows][M][2] K_{imp} (slice-relative)
  const float *mx;       // [n_rows][n_det][REC] <h_m|h_m'>_k (slice-relative)
  float z_scale;         // accumulator -> Z scale (times 1 / *g_scale)
  const float *g_scale;
  float rank_tol;
  unsigned long long *keys;  // [n_rows][n_det] out: (ln L^ML bits << 32) | ~(t n_phi + o), zeroed
  int *status;
  unsigned long long wait_ns;
};
struct PreselOut {
  double max_inco, threshold;
  long long arg_i, n_selected;
};
// returns a cudaError_t
// pol: a polarisation-resolved bank (time-grid operand from launch_presel_pol_pack, 32 columns per tile)
int launch_presel(const CUtensorMap &mapG, const CUtensorMap &mapBank, const PreselParams &p, bool bf16, bool split,
                  bool per_mode, bool pol, int n_sms, cudaStream_t st);
void launch_presel_finish(int64_t n, int D, int n_phi, double delta, const unsigned long long *keys, float *ml,
                          int *arg_ot, double *inco, unsigned long long *max_bits /*zeroed*/, int64_t *sel,
                          PreselOut *out, cudaStream_t st);

// Pre-selection of a polarisation-resolved bank, FP32 on the CUDA cores
// (kernel_presel_pol.cu): the same keys as launch_presel, then launch_presel_finish.
struct PreselPolArgs {
  int64_t n_rows;            // rows of the slice
  int64_t row0, bank_rows;   // first bank row of the slice, rows of the bank
  int n_det, n_t, n_tpad, n_phi, n_modes, n_bins, kpad;
  int mode_m[MAXM];
  const float *master;       // FP32 master [M][bank_rows][kpad], rows [Re h+ | Im h+ | Re hx | Im hx | 0]
  const float2 *G;           // [n_gcomp][n_det][n_bins][n_tpad] time-grid operand c_kjb e^{-2 pi i f_b t_kt},
                             // times innermost so that a warp's threads (times) read consecutive words
  int n_gcomp;               // 1 (one operand for every component), or 2 n_modes with relative binning (j = 2m + p)
  const float *mx;           // [n_rows][n_det][REC_P] overlap records (slice-relative)
  float rank_tol;
  unsigned long long *keys;  // [n_rows][n_det] out, zeroed
};
void launch_presel_pol(const PreselPolArgs &a, cudaStream_t st);
// The tensor-core pre-selection's time-grid operand for a polarisation-resolved
// bank: rows 4c + 2p + part (c = detector-time column), polarisation block p of
// [Re | Im | Re | Im] along K holding the column's real-ified G, the other zero.
// Gp: [2][2 n_cols][B] FP32 scratch; G32 [n_cols][B]; out and scale as launch_prep's pack.
// GT [n_mat][B][T] = G [n_mat][T][B] transposed (the FP32 kernel's operand layout).
void launch_transpose_G(int64_t n_mat, int T, int B, const float2 *G, float2 *GT, cudaStream_t st);
void launch_presel_pol_pack(int64_t n_cols, int B, int Kpad, const float2 *G32, float2 *Gp, const float *gmax,
                            int kind, int planes, void *out, float *scale_out, cudaStream_t st);

// Relative-binning weights (App. A): kernel_rb.cu.  w_dh [D][M][B], w_hh [D][M][M][B].
void launch_rb_weights(int D, int M, int64_t N, const double *ff, const double *dff, const double *psd,
                       const double2 *data, const double2 *h0, const double *t0, int B, const int64_t *node,
                       double2 *w_dh, double2 *w_hh, int *status, cudaStream_t st);

// Posterior samples of a finished event: kernel_sample.cu.
struct SampleArgs {
  int64_t n_int, n_ext;         // slice rows, extrinsic samples
  int n_det, n_modes, n_bins, n_phi;
  int mode_m[MAXM];
  int64_t i_base, bank_rows;    // first bank row of the slice, rows of the bank
  int kpad;
  const float *master;          // bank FP32 master [M][bank_rows][kpad] ([re | im | pad])
  const double *f, *w;          // [B]
  const double *psd;            // [D][B] (plain quadrature)
  const double2 *data;          // [D][B]
  const double2 *rb_dh, *rb_hh; // relative-binning weights, or null
  const double *t;              // [E][D]
  const double2 *R;             // [E][D][M]
  const double *F;              // [E][D][2] antenna patterns (n_pol = 2)
  int n_pol;                    // 2: polarisation-resolved bank (master rows [h+ | hx])
  const double *lw_ext;         // [E] or null
  const double *ln_p_int;       // [n_int] ln sum_{e,o} p_ieo
  const float *lnl;             // [n_int][n_ext] stored ln Lbar_ie
  double threshold;             // the event's ML cut (-inf: none)
  float u_min;
  const float4 *dm_table;
  int *status;
};
// cdf: n_int doubles of scratch; outputs may be null
void launch_sample(const SampleArgs &a, int64_t n, const double *uni, double *cdf, int64_t *i_out, int64_t *e_out,
                   int32_t *o_out, double *d_out, cudaStream_t st);

// Pilot tiles of a screening launch (cut on, grid order): a spread-out 1/48
// of the event's work tiles is screened first, so that the running maximum,
// and with it the cut's threshold, is near its final value before the bulk of
// the tiles (which then skip almost every pair on their bounds) is screened.
// They form a grid of evenly spread bank tiles by up to TC_PILOT_COLS evenly
// spread extrinsic tiles, the bank tile slowest, so that each operand tile
// the pilots read comes from memory once.  The band-order sweep skips them
// (their first pass wrote every output, with a lower threshold).
constexpr int TC_PILOT_COLS = 8;
// pair: the work items are 256-row pair tiles of a CTA pair.
__host__ __device__ inline int tc_pilot_tiles(const TcEvent &w, int tev, bool pair = false) {
  if (!w.P.screen_ml || w.P.gemm_only || w.P.cut_delta <= 0.f || w.P.lnl_tile) return 0;
  const int rs = tev / TC_TE;
  const int t = (pair ? (w.n_itile + 1) / 2 : w.n_itile) * ((w.n_etile + rs - 1) / rs);
  return t >= 96 ? t / 48 : 0;
}

// Work items of one event in a launch of tile width tev (grid order).
__host__ __device__ inline int tc_work_items(const TcEvent &w, int tev, bool pair = false) {
  const int rs = tev / TC_TE;
  return tc_pilot_tiles(w, tev, pair) + (pair ? (w.n_itile + 1) / 2 : w.n_itile) * ((w.n_etile + rs - 1) / rs);
}

// Tensor-map encoding through the driver entry point.
int encode_tmap_kblocks(CUtensorMap *map, CUtensorMapDataType dt, void *base, uint64_t rows, uint64_t n_kb,
                        uint64_t row_bytes, uint32_t box_rows, uint32_t box_kb);
int tc_kblocks_per_stage();

}  // namespace dotpe
