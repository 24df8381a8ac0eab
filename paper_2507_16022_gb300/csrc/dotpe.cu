// dotpe C ABI and runtime: context, bank residency, event admission by HBM
// footprint, concurrent event slots (one CUDA stream each), results.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "kernels.h"

namespace dotpe {

static thread_local std::string g_last_error;

static int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define CUDA_OR_FAIL(expr)                                                                         \
  do {                                                                                             \
    cudaError_t e_ = (expr);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return fail(e_ == cudaErrorMemoryAllocation ? DOTPE_E_NOMEM : DOTPE_E_DEVICE, "%s: %s (%s:%d)", \
                  #expr, cudaGetErrorString(e_), __FILE__, __LINE__);                              \
  } while (0)

static int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Records `ev` on `st`; inside a stream capture as an event-record node of the
// graph (a plain record there only orders the captured work and is never
// executed, so the host could not query or time the event afterwards).
static cudaError_t record(cudaEvent_t ev, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) return e;
  return cudaEventRecordWithFlags(ev, st, cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal
                                                                               : cudaEventRecordDefault);
}

// Carves one allocation into 256-byte aligned pieces.
// NVTX range over a host scope (the enqueueing of one stage of an event or a
// call); profilers that record NVTX show the stages by name.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

struct Carver {
  size_t off = 0;
  template <typename T>
  size_t take(size_t n) {
    size_t o = off;
    off = align256(off + n * sizeof(T));
    return o;
  }
};

static bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Row records <h_m|h_m'>_d of every bank row for one noise PSD (Eq. hh_ieo):
// they depend on the bank and on omega = 4w/S only, so events that share a PSD
// share them.  Kept per bank, keyed by a hash of (n_det, PSD values).
struct XEntry {
  uint64_t key = 0;
  int D = 0;
  float *mx = nullptr;  // [I][D][16]
  size_t bytes = 0;
  cudaEvent_t ready = nullptr;  // recorded after the records are written
  int refs = 0;                 // events that may still read them
  int64_t last = 0;             // last use (LRU)
};
constexpr int XCACHE_MAX = 4;  // entries per bank

struct Bank {
  uint64_t id = 0;
  int64_t I = 0;
  int M = 0, B = 0, Kpad = 0;
  int mode_m[MAXM] = {0, 0, 0, 0};
  int n_pol = 1;  // 2: polarisation-resolved bank, rows [Re h+ | Im h+ | Re hx | Im hx | pad]
  double *f = nullptr, *w = nullptr, *lw = nullptr;  // device
  float *master = nullptr;                           // [M][I][Kpad]
  __nv_bfloat16 *bf = nullptr;                       // [2][M][I][Kpad] hi, lo
  __half *hf = nullptr;                              // [2][M][I][Kpad] hi, lo
  float a_scale = 1.f;
  float2 *pol = nullptr;  // [I][M][2] polarisation factors K_{imp} (pre-selection), or null
  void *block = nullptr;
  size_t bytes = 0;
  int refs = 0;
  std::vector<XEntry *> xcache;
};

struct Event {
  uint64_t id = 0;
  Bank *bank = nullptr;
  int state = DOTPE_STATE_QUEUED;
  int64_t i0 = 0, NI = 0, NE = 0;
  int64_t block_rows = 0;  // rows per streamed bank block (0: the whole slice)
  uint64_t group = 0;      // batch of dotpe_batch_submit (0: none)
  uint64_t psd_key = 0;    // hash of (n_det, PSD values): the cross-term cache key
  XEntry *xent = nullptr;  // cross terms in use
  std::string launch_error;  // why the launch failed on the host (state FAILED, device status 0)
  float frozen_max = -1.f;   // >= 0: the cut's maximum is fixed at this value (block recomputation)
  bool owns_inputs = true;   // false: the inputs belong to another event
  int D = 0, nphi = 0, prec = 0, flags = 0;
  double u_min = 0, cut = 0;
  bool has_lwe = false;
  // inputs: device copy made at submit
  void *in_block = nullptr;
  size_t in_bytes = 0;
  double *psd = nullptr, *t = nullptr, *lwe = nullptr;
  double2 *data = nullptr, *R = nullptr;
  double2 *rb_dh = nullptr, *rb_hh = nullptr;  // relative-binning weights (App. A), or null
  double *F = nullptr;  // [E][D][2] antenna patterns (polarisation-resolved bank), or null
  void *in_stage = nullptr;  // pinned host staging of host inputs
  size_t stage_bytes = 0;
  cudaEvent_t ev_inputs = nullptr, ev_start = nullptr, ev_end = nullptr, ev_k0 = nullptr, ev_k1 = nullptr,
              ev_ks = nullptr;
  // results kept until release
  void *keep_block = nullptr;
  size_t keep_bytes = 0;
  double *ln_p_int = nullptr, *ln_p_ext = nullptr;
  float *lnl_tile = nullptr, *ml_tile = nullptr;
  ReduceOut *d_out = nullptr;
  ReduceOut *h_out = nullptr;  // pinned
  size_t scratch_bytes = 0;
  bool want_hb = false;  // admitted with room for the tensor-core <h|h> bound of its screen
  int slot = -1;
  int64_t t_submit = 0, t_admit = 0;
  volatile int64_t t_done = 0;
  float device_ms = -1.f, prep_ms = -1.f, fused_ms = -1.f, refine_ms = -1.f;
  int refined = -1;  // tiles refined (mixed precision)
};

}  // namespace dotpe

struct dotpe_ctx {
  int device = 0;
  int n_sms = 0;
  char name[256] = {0};
  uint64_t budget = 0, used = 0;
  std::vector<cudaStream_t> streams;
  std::vector<int> slot_busy;  // events in flight on each slot's stream
  cudaStream_t main_stream = nullptr, input_stream = nullptr;
  float4 *dm_table = nullptr;
  std::mutex mu;
  std::unordered_map<uint64_t, dotpe::Bank *> banks;
  std::unordered_map<uint64_t, dotpe::Event *> events;
  std::deque<uint64_t> queue;
  uint64_t next_id = 1, next_group = 1;
  int max_batch = 1;     // queued events one fused launch may take (continuous batching)
  bool use_graphs = true;  // batches run as captured CUDA graphs
  bool autotune = false;   // time L2 band widths on first use of a shape
  std::unordered_map<std::string, int> band_cache;                        // shape key -> band
  std::unordered_map<std::string, int> tev_cache;                         // shape key -> screening tile width
  std::unordered_map<std::string, bool> pair_cache;                       // shape key -> 64-sample tiles on CTA pairs
  bool wide_tiles = true;  // 64-sample tiles for screening / GEMM-only launches of mode banks
  bool pair_tiles = true;  // those tiles on CTA pairs (single events)
  std::vector<std::unordered_map<std::string, cudaGraphExec_t>> graphs;  // per slot
  double l2_band_bytes = 0;  // extrinsic operand kept in L2 per sweep of the bank
  // completion callbacks -> admission worker
  std::mutex cb_mu;
  std::condition_variable cv;
  std::unordered_map<uint64_t, int64_t> done_ns;
  bool stop = false;
  std::thread worker;
};

namespace dotpe {

struct DoneArg {
  dotpe_ctx *ctx;
  uint64_t id;
};

// Host callback at the end of an event's stream work: records the completion
// time and wakes the admission worker.  It touches no CUDA API and not the
// Event itself (which the caller may release concurrently).
static void CUDART_CB mark_done(void *p) {
  DoneArg *a = (DoneArg *)p;
  {
    std::lock_guard<std::mutex> lk(a->ctx->cb_mu);
    a->ctx->done_ns[a->id] = now_ns();
  }
  a->ctx->cv.notify_all();
  delete a;
}

// ---------------------------------------------------------------------------
// footprint of one event's device scratch (freed when the event completes)
// ---------------------------------------------------------------------------
struct ScratchLayout {
  size_t c, omega, fh, fl, th, tl, Rf, qx, G32, gmax, gscale, sqrt_dd, gpack, mx, tile_part, tile_ml, tile_arg,
      tile_npass, row_part, col_part, ml_running, ml_refine, list, n_list, n_list_total, sel_counts, sep, n_cand, acc,
      acc_col, status, red, hb, total;
  size_t hb_bytes;     // scratch of the tensor-core <h|h> bound (0: the screen forms it itself)
  int64_t block_rows;  // bank rows per streamed block (the whole slice when not streamed)
  int n_itile, n_etile, pack_kind, pack_planes, TI, TE;  // n_itile: tiles of one block
};

static bool prec_split(int p) { return p == DOTPE_PREC_BF16X3 || p == DOTPE_PREC_FP16X3 || p == DOTPE_PREC_MIXED; }
static bool prec_bf16(int p) { return p == DOTPE_PREC_BF16 || p == DOTPE_PREC_BF16X3; }

// Screening error scale kappa*u of a single fp16 pass (u = 2^-11, kappa = 2).
static const float MIXED_MARGIN_K = 2.0f * 0.00048828125f;
// With the cut off, tiles whose screened best ln L^ML lies this far below the
// maximum keep their screened values (their share of Z is below e^-30 each).
static const float MIXED_FAR_WINDOW = 30.0f;

// The screening pass of a mixed event with the cut on reads a per-pair bound
// of <h|h> from the tensor-core pass when its buffer (2 bytes per pair of a
// bank block) stays under this size (and the launch unit's scratch with the
// bounds fits the HBM budget).
static const size_t HB_MAX_BYTES = (size_t)8 << 30;

static ScratchLayout scratch_layout(const Event &e, bool want_hmin = false) {
  ScratchLayout L{};
  const Bank &b = *e.bank;
  const int64_t D = e.D, B = b.B, M = b.M, E = e.NE, Kp = b.Kpad;
  const bool simt = (e.prec == DOTPE_PREC_FP32);
  L.block_rows = (e.block_rows > 0 && e.block_rows < e.NI) ? e.block_rows : e.NI;
  const int64_t NI = L.block_rows;  // per-block arrays
  L.TI = simt ? SIMT_TI : TC_TI;
  L.TE = simt ? SIMT_TE : TC_TE;
  L.n_itile = (int)((NI + L.TI - 1) / L.TI);
  L.n_etile = (int)((E + L.TE - 1) / L.TE);
  L.pack_kind = simt ? 0 : (prec_bf16(e.prec) ? 1 : 2);
  L.pack_planes = prec_split(e.prec) ? 2 : 1;
  size_t elem = (L.pack_kind == 0) ? 4 : 2;
  const int64_t T = (int64_t)L.n_itile * L.n_etile;
  Carver c;
  L.c = c.take<float2>(D * M * b.n_pol * B);  // data weights per (mode, polarisation) component
  L.omega = c.take<float>(D * B);
  L.fh = c.take<float>(B);
  L.fl = c.take<float>(B);
  L.th = c.take<float>(E * D);
  L.tl = c.take<float>(E * D);
  L.Rf = c.take<float2>(E * D * M);
  L.qx = c.take<float>(E * D * REC);
  L.G32 = c.take<float2>(M * E * B * (b.n_pol == 2 ? 2 : 1));
  L.gmax = c.take<float>(1);
  L.gscale = c.take<float>(1);
  L.sqrt_dd = c.take<float>(1);
  L.gpack = c.take<uint8_t>((size_t)L.pack_planes * M * 2 * E * Kp * elem);
  L.mx = c.take<float>(NI * D * (b.n_pol == 2 ? REC_P : REC));
  L.tile_part = c.take<float4>(T);
  L.tile_ml = c.take<float>(T);
  L.tile_arg = c.take<long long>(T);
  L.tile_npass = c.take<int>(T);
  L.row_part = c.take<float2>((size_t)L.n_etile * NI);
  L.col_part = c.take<float2>((size_t)L.n_itile * E);
  L.ml_running = c.take<float>(1);
  const bool mixed = (e.prec == DOTPE_PREC_MIXED);
  L.ml_refine = c.take<float>(1);
  L.list = c.take<int2>(mixed ? T : 0);
  L.n_list = c.take<int>(1);
  L.n_list_total = c.take<int>(1);
  L.sep = c.take<int>(1);
  L.n_cand = c.take<unsigned long long>(2);
  L.sel_counts = c.take<int>(mixed ? select_count_blocks((int)T) : 0);
  L.acc = c.take<EvAcc>(1);
  L.acc_col = c.take<double2>(E);
  L.status = c.take<int>(1);
  L.red = c.take<uint8_t>(reduce_scratch_bytes());
  L.hb_bytes = 0;
  if (want_hmin && e.prec == DOTPE_PREC_MIXED && e.cut > 0 && !(e.flags & DOTPE_FLAG_STORE_LNL) && b.n_pol == 1) {
    const size_t hb = hb_scratch_bytes(NI, E);
    if (hb <= HB_MAX_BYTES) L.hb_bytes = hb;
  }
  L.hb = c.take<uint8_t>(L.hb_bytes);
  L.total = c.off;
  return L;
}

static size_t keep_bytes_of(const Event &e) {
  size_t k = align256(sizeof(ReduceOut)) + align256(e.NI * 8) + align256(e.NE * 8);
  if (e.flags & DOTPE_FLAG_STORE_LNL) k += 2 * align256((size_t)e.NI * e.NE * 4);
  return k;
}

// ---------------------------------------------------------------------------
// launching admitted events
// ---------------------------------------------------------------------------
// Device-side plan of one admitted event: its scratch, the prep arguments, the
// epilogue parameters, its tensor-core work record and the reduction arguments.
struct EventRun {
  ScratchLayout L;
  uint8_t *scr = nullptr;
  PrepArgs pa;
  EpiParams P;
  TcWork W;
  ReduceArgs ra;
  bool mixed = false;
};

// The bank operand map and the shape common to every event of a launch.
static int tc_launch_of(dotpe_ctx *ctx, const Bank &b, int prec, TcLaunch &T) {
  memset(&T, 0, sizeof(T));
  const bool bf = prec_bf16(prec);
  const int64_t a_rows = 2 * (int64_t)b.M * b.I;
  if (a_rows >= (1ll << 31)) return fail(DOTPE_E_UNSUPPORTED, "bank too large for 32-bit TMA coordinates");
  CUtensorMapDataType dt = bf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  void *abase = bf ? (void *)b.bf : (void *)b.hf;
  if (encode_tmap_kblocks(&T.mapA, dt, abase, a_rows, b.Kpad / 64, (uint64_t)b.Kpad * 2, TC_TI,
                          tc_kblocks_per_stage()))
    return fail(DOTPE_E_DEVICE, "cuTensorMapEncodeTiled failed (bank)");
  T.C.kb = b.Kpad / 64;
  T.C.a_plane_rows = b.M * (int)b.I;
  T.C.a_mode_rows = (int)b.I;
  T.C.n_modes = b.M;
  T.bf16 = bf;
  T.split = prec_split(prec) && prec != DOTPE_PREC_MIXED;
  T.sep = T.split;  // full split runs keep the low-order terms apart (precision first)
  T.pair = ctx->pair_tiles;  // taken by single-event launches of 64-sample tiles
  T.consec = true;
  for (int m = 1; m < b.M; ++m)
    if (b.mode_m[m] != b.mode_m[m - 1] + 1) T.consec = false;
  T.pol = (b.n_pol == 2);
  T.n_sms = ctx->n_sms;
  return DOTPE_OK;
}

// L2 band width of an event: tuned value if the autotuner has one, else the default.
static int event_band(dotpe_ctx *ctx, const Event &e, const ScratchLayout &L, bool split);

// Device allocations of an event and every pointer of its plan (no launches).
static int event_alloc(dotpe_ctx *ctx, Event &e, cudaStream_t st, EventRun &R) {
  Bank &b = *e.bank;
  R.L = scratch_layout(e, e.want_hb);
  const ScratchLayout &L = R.L;
  e.scratch_bytes = L.total;
  CUDA_OR_FAIL(cudaStreamWaitEvent(st, e.ev_inputs, 0));
  CUDA_OR_FAIL(cudaMallocAsync((void **)&R.scr, L.total, st));
  e.keep_bytes = keep_bytes_of(e);
  uint8_t *keep = nullptr;
  CUDA_OR_FAIL(cudaMallocAsync((void **)&keep, e.keep_bytes, st));
  e.keep_block = keep;
  {
    Carver c;
    e.d_out = (ReduceOut *)(keep + c.take<ReduceOut>(1));
    e.ln_p_int = (double *)(keep + c.take<double>(e.NI));
    e.ln_p_ext = (double *)(keep + c.take<double>(e.NE));
    if (e.flags & DOTPE_FLAG_STORE_LNL) {
      e.lnl_tile = (float *)(keep + c.take<float>((size_t)e.NI * e.NE));
      e.ml_tile = (float *)(keep + c.take<float>((size_t)e.NI * e.NE));
    }
  }
  uint8_t *scr = R.scr;
  int *status = (int *)(scr + L.status);
  PrepArgs &pa = R.pa;
  pa.D = e.D; pa.B = b.B; pa.M = b.M; pa.Kpad = b.Kpad; pa.E = e.NE;
  pa.f = b.f; pa.w = b.w; pa.psd = e.psd; pa.data = e.data; pa.t = e.t; pa.R = e.R;
  pa.rb_dh = e.rb_dh; pa.rb_hh = e.rb_hh;
  pa.n_pol = b.n_pol; pa.F = e.F;
  pa.c = (float2 *)(scr + L.c);
  pa.omega = (float *)(scr + L.omega);
  pa.fh = (float *)(scr + L.fh);
  pa.fl = (float *)(scr + L.fl);
  pa.th = (float *)(scr + L.th);
  pa.tl = (float *)(scr + L.tl);
  pa.Rf = (float2 *)(scr + L.Rf);
  pa.qx = (float *)(scr + L.qx);
  pa.G32 = (float2 *)(scr + L.G32);
  pa.gmax = (float *)(scr + L.gmax);
  pa.gpack = scr + L.gpack;
  pa.pack_kind = L.pack_kind;
  pa.pack_planes = L.pack_planes;
  pa.gscale = (float *)(scr + L.gscale);
  pa.sqrt_dd = (float *)(scr + L.sqrt_dd);
  pa.status = status;

  EpiParams &P = R.P;
  memset(&P, 0, sizeof(P));
  P.n_modes = b.M;
  P.n_det = e.D;
  P.n_phi = e.nphi;
  P.n_pol = b.n_pol;
  for (int m = 0; m < MAXM; ++m) P.mode_m[m] = m < b.M ? b.mode_m[m] : 0;
  P.npair = b.M * (b.M - 1) / 2;
  {
    int p = 0;
    for (int a = 1; a < MAXM; ++a)
      for (int c = 0; c < a; ++c, ++p) P.pdelta[p] = (a < b.M) ? (b.mode_m[a] - b.mode_m[c]) : 0;
  }
  P.consec = 1;
  for (int m = 1; m < b.M; ++m)
    if (b.mode_m[m] != b.mode_m[m - 1] + 1) P.consec = 0;
  P.u_min = (float)e.u_min;
  P.cut_delta = (float)(e.cut > 0 ? e.cut : 0.0);
  P.ln_nphi = (float)std::log((double)e.nphi);
  P.n_ext = e.NE;
  P.mx = (float *)(scr + L.mx);
  P.qx = pa.qx;
  P.lw_ext = e.has_lwe ? e.lwe : nullptr;
  P.dm_table = ctx->dm_table;
  P.ml_running = (float *)(scr + L.ml_running);
  P.track_max = (P.cut_delta > 0.f && e.frozen_max < 0.f) ? 1 : 0;
  P.sqrt_dd = pa.sqrt_dd;
  P.tile_part = (float4 *)(scr + L.tile_part);
  P.row_part = (float2 *)(scr + L.row_part);
  P.col_part = (float2 *)(scr + L.col_part);
  P.tile_ml = (float *)(scr + L.tile_ml);
  P.tile_arg = (long long *)(scr + L.tile_arg);
  P.tile_npass = (int *)(scr + L.tile_npass);
  P.status = status;
  P.gemm_only = (e.flags & DOTPE_FLAG_GEMM_ONLY) ? 1 : 0;
  P.test_stall = (e.flags & DOTPE_FLAG_TEST_STALL) ? 1 : 0;
  P.wait_ns = P.test_stall ? 250000000ull : 4000000000ull;
  R.mixed = (e.prec == DOTPE_PREC_MIXED);
  if (e.prec != DOTPE_PREC_FP32) {
    P.z_scale = 1.f / (b.a_scale * (prec_bf16(e.prec) ? 1.f : FP16_OPERAND_SCALE));
    P.g_scale = pa.gscale;
    TcWork &W = R.W;
    memset(&W, 0, sizeof(W));
    const bool bf = prec_bf16(e.prec);
    const int64_t b_rows = (int64_t)L.pack_planes * b.M * 2 * e.NE;
    if (b_rows >= (1ll << 31)) return fail(DOTPE_E_UNSUPPORTED, "n_ext too large for 32-bit TMA coordinates");
    CUtensorMapDataType dt = bf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    if (encode_tmap_kblocks(&W.mapB, dt, pa.gpack, b_rows, b.Kpad / 64, (uint64_t)b.Kpad * 2, 2 * TC_TE,
                            tc_kblocks_per_stage()))
      return fail(DOTPE_E_DEVICE, "cuTensorMapEncodeTiled failed (extrinsic operand)");
    // 128-row boxes for 64-sample tiles (mode banks)
    if (b.n_pol != 2 && encode_tmap_kblocks(&W.mapB64, dt, pa.gpack, b_rows, b.Kpad / 64, (uint64_t)b.Kpad * 2,
                                            4 * TC_TE, tc_kblocks_per_stage()))
      return fail(DOTPE_E_DEVICE, "cuTensorMapEncodeTiled failed (extrinsic operand, 128-row boxes)");
    W.n_etile = L.n_etile;
    W.band = event_band(ctx, e, L, prec_split(e.prec));
    W.b_plane_rows = b.M * 2 * (int)e.NE;
    W.b_mode_rows = 2 * (int)e.NE;
  } else {
    P.z_scale = 1.f;
    P.g_scale = nullptr;
  }

  ReduceArgs &ra = R.ra;
  memset(&ra, 0, sizeof(ra));
  ra.n_ext = e.NE;
  ra.n_int_total = e.NI;
  ra.n_etile = L.n_etile;
  ra.n_phi = e.nphi;
  ra.tile_part = P.tile_part;
  ra.row_part = P.row_part;
  ra.col_part = P.col_part;
  ra.tile_ml = P.tile_ml;
  ra.tile_arg = P.tile_arg;
  ra.tile_npass = P.tile_npass;
  ra.ml_running = R.mixed ? (const float *)(scr + L.ml_refine) : P.ml_running;
  ra.cut_delta = P.cut_delta;
  ra.ln_p_int = e.ln_p_int;
  ra.ln_p_ext = e.ln_p_ext;
  ra.acc = (EvAcc *)(scr + L.acc);
  ra.acc_col = (double2 *)(scr + L.acc_col);
  ra.status = status;
  ra.scratch = scr + L.red;
  ra.out = e.d_out;
  ra.n_refined = R.mixed ? (const int *)(scr + L.n_list) : nullptr;
  ra.n_cand = R.mixed ? (const unsigned long long *)(scr + L.n_cand) : nullptr;
  return DOTPE_OK;
}

// Stream work before the fused kernel: zeroed scalars, data weights, extrinsic operand.
static int event_begin(Event &e, EventRun &R, cudaStream_t st) {
  CUDA_OR_FAIL(cudaMemsetAsync(R.scr + R.L.gmax, 0, 4, st));
  if (e.frozen_max >= 0.f)
    CUDA_OR_FAIL(cudaMemcpyAsync(R.scr + R.L.ml_running, &e.frozen_max, 4, cudaMemcpyHostToDevice, st));
  else
    CUDA_OR_FAIL(cudaMemsetAsync(R.scr + R.L.ml_running, 0, 4, st));
  CUDA_OR_FAIL(cudaMemsetAsync(R.scr + R.L.status, 0, 4, st));
  CUDA_OR_FAIL(cudaMemsetAsync(R.scr + R.L.n_cand, 0, 16, st));
  CUDA_OR_FAIL(record(e.ev_start, st));
  launch_prep(R.pa, st);
  return DOTPE_OK;
}

// Rows [r0, r0 + nr) of the slice as the current bank block of the plan.
static void event_block(dotpe_ctx *ctx, Event &e, EventRun &R, int64_t r0, int64_t nr, cudaStream_t st) {
  Bank &b = *e.bank;
  if (e.xent) {
    R.P.mx = e.xent->mx + (e.i0 + r0) * e.D * (b.n_pol == 2 ? REC_P : REC);
  } else if (b.n_pol == 2) {
    launch_cross_terms_pol(nr, e.i0 + r0, b.I, b.M, e.D, b.B, b.Kpad, b.mode_m, b.master, R.pa.omega, e.rb_hh,
                           (float *)(R.scr + R.L.mx), ctx->n_sms, st);
  } else {
    launch_cross_terms(nr, e.i0 + r0, b.I, b.M, e.D, b.B, b.Kpad, b.master, R.pa.omega, e.rb_hh,
                       (float *)(R.scr + R.L.mx), ctx->n_sms, st);
  }
  R.P.n_int = nr;
  R.P.i_base = e.i0 + r0;
  R.P.lw_int = b.lw ? b.lw + e.i0 + r0 : nullptr;
  R.P.lnl_tile = e.lnl_tile ? e.lnl_tile + r0 * e.NE : nullptr;
  R.P.ml_tile = e.ml_tile ? e.ml_tile + r0 * e.NE : nullptr;
  R.W.n_itile = (int)((nr + TC_TI - 1) / TC_TI);
  R.W.a_row0 = (int)(e.i0 + r0);
  R.ra.n_int = nr;
  R.ra.row_offset = r0;
  R.ra.n_itile = (int)((nr + R.L.TI - 1) / R.L.TI);
}

// Screening variant of an event's parameters (mixed precision).
static EpiParams screen_params(const EventRun &R) {
  EpiParams Ps = R.P;
  Ps.track_max = 1;
  Ps.screen_ml = (R.P.cut_delta > 0.f) ? 1 : 0;
  Ps.margin_k = MIXED_MARGIN_K;
  Ps.n_cand = (unsigned long long *)(R.scr + R.L.n_cand);
  return Ps;
}

static SelectEvent select_event_of(const EventRun &R) {
  SelectEvent v;
  v.tile_ml = R.P.tile_ml;
  v.n_itile = R.W.n_itile;
  v.n_etile = R.W.n_etile;
  v.band = R.W.band;
  v.ml_screen = R.P.ml_running;
  v.sqrt_dd = R.pa.sqrt_dd;
  v.window = (R.P.cut_delta > 0.f) ? R.P.cut_delta : MIXED_FAR_WINDOW;
  v.margin_k = MIXED_MARGIN_K;
  v.sep_ml = SEP_ML * (R.pa.Kpad > 1024 ? 1024.f / (float)R.pa.Kpad : 1.f);
  v.ml_refine = (float *)(R.scr + R.L.ml_refine);
  v.n_refined = (int *)(R.scr + R.L.n_list);
  return v;
}

// Refinement variant: threshold frozen at (screened maximum - margin) - cut_delta.
static EpiParams refine_params(const EventRun &R) {
  EpiParams Pf = R.P;
  Pf.ml_running = (float *)(R.scr + R.L.ml_refine);
  Pf.track_max = 0;
  return Pf;
}

static std::string band_key(const Event &e, const ScratchLayout &L, bool split);

// Tile width of a single-pass launch: 64-sample tiles where the launch writes
// no marginal partials (a screening pass with the cut on, or GEMM-only) over a
// mode bank, unless the context asks for 32-sample tiles; the autotuner's
// choice for the shape where it has one.
static int launch_tev(dotpe_ctx *ctx, const Event &e, const ScratchLayout &L, const EpiParams &P, bool split) {
  if (!ctx->wide_tiles || split || e.bank->n_pol == 2 || P.lnl_tile) return 32;
  if (!(P.gemm_only || P.screen_ml)) return 32;
  auto it = ctx->tev_cache.find(band_key(e, L, prec_split(e.prec)));
  return it != ctx->tev_cache.end() ? it->second : 64;
}

// Whether a single event's 64-sample tiles run on CTA pairs: the autotuner's
// choice for the shape where it has one, else the context's default.
static bool launch_pair(dotpe_ctx *ctx, const Event &e, const ScratchLayout &L) {
  if (!ctx->pair_tiles) return false;
  auto it = ctx->pair_cache.find(band_key(e, L, prec_split(e.prec)));
  return it != ctx->pair_cache.end() ? it->second : true;
}

// The <h|h> bound of every pair of the current bank block on the tensor cores,
// for the 64-sample screen P (when the event's scratch has room for it).
static int hh_bound_pass(dotpe_ctx *ctx, const Event &e, EventRun &R, EpiParams &P, cudaStream_t st) {
  if (R.L.hb_bytes == 0) return DOTPE_OK;
  HbDelta dl;
  for (int p = 0; p < NPAIR; ++p) dl.pdelta[p] = R.P.pdelta[p];
  __nv_bfloat16 *hmin = nullptr;
  if (launch_hh_bound(R.P.n_int, e.NE, e.D, dl, R.P.mx, R.pa.qx, R.scr + R.L.hb, &hmin, ctx->n_sms, R.P.status,
                      st) != 0)
    return fail(DOTPE_E_DEVICE, "<h|h> bound launch failed: %s", cudaGetErrorString(cudaGetLastError()));
  P.hmin = hmin;
  P.hmin_ld = hb_ld(e.NE);
  return DOTPE_OK;
}

// The fused kernel(s) of the current block of one event (mixed: screen,
// selection, refinement over the event's own list).
static int event_fused(dotpe_ctx *ctx, Event &e, EventRun &R, bool last_block, cudaStream_t st) {
  Bank &b = *e.bank;
  if (e.prec == DOTPE_PREC_FP32) {
    SimtArgs sg;
    sg.A = b.master;
    sg.Bm = (const float *)R.pa.gpack;
    sg.I_bank = b.I;
    sg.Kpad = b.Kpad;
    sg.K = 2 * b.n_pol * b.B;
    launch_simt(sg, R.P, st);
    return DOTPE_OK;
  }
  TcLaunch T;
  int rc = tc_launch_of(ctx, b, e.prec, T);
  if (rc != DOTPE_OK) return rc;
  TcWork W = R.W;
  if (!R.mixed) {
    W.P = R.P;
    T.tev = launch_tev(ctx, e, R.L, W.P, T.split);
    T.pair = launch_pair(ctx, e, R.L);
    int r = launch_tc(T, &W, 1, nullptr, nullptr, st);
    if (r != 0) return fail(DOTPE_E_DEVICE, "tcgen05 kernel launch failed: %s", cudaGetErrorString((cudaError_t)r));
    return DOTPE_OK;
  }
  W.P = screen_params(R);
  T.tev = launch_tev(ctx, e, R.L, W.P, false);
  T.pair = launch_pair(ctx, e, R.L);
  if (T.tev == 64 && (rc = hh_bound_pass(ctx, e, R, W.P, st)) != DOTPE_OK) return rc;
  int r = launch_tc(T, &W, 1, nullptr, nullptr, st);
  if (r != 0) return fail(DOTPE_E_DEVICE, "tcgen05 kernel launch failed: %s", cudaGetErrorString((cudaError_t)r));
  if (last_block) CUDA_OR_FAIL(record(e.ev_ks, st));
  T.tev = 32;
  SelectBatch sb;
  memset(&sb, 0, sizeof(sb));
  sb.ev[0] = select_event_of(R);
  sb.begin[0] = 0;
  sb.begin[1] = R.W.n_itile * R.W.n_etile;
  sb.n = 1;
  sb.list = (int2 *)(R.scr + R.L.list);
  sb.n_list = (int *)(R.scr + R.L.n_list_total);
  sb.counts = (int *)(R.scr + R.L.sel_counts);
  sb.sep = (int *)(R.scr + R.L.sep);
  launch_select(sb, st);
  CUDA_OR_FAIL(cudaGetLastError());
  W.P = refine_params(R);
  // two variants, gated per event by its screened maximum: the shared
  // accumulator, or the separate low-order accumulator above SEP_ML
  T.split = true;
  T.gate = sb.sep;
  for (int want = 0; want < 2; ++want) {
    T.sep = want == 1;
    T.gate_want = want;
    r = launch_tc(T, &W, 1, sb.list, sb.n_list, st);
    if (r != 0) return fail(DOTPE_E_DEVICE, "tcgen05 kernel launch failed: %s", cudaGetErrorString((cudaError_t)r));
  }
  return DOTPE_OK;
}

// After the last block: evidence, copy to the host, completion callback.
static int event_end(dotpe_ctx *ctx, Event &e, EventRun &R, cudaStream_t st) {
  launch_reduce_final(R.ra, st);
  CUDA_OR_FAIL(cudaGetLastError());
  CUDA_OR_FAIL(cudaMemcpyAsync(e.h_out, e.d_out, sizeof(ReduceOut), cudaMemcpyDeviceToHost, st));
  CUDA_OR_FAIL(record(e.ev_end, st));
  CUDA_OR_FAIL(cudaLaunchHostFunc(st, mark_done, new DoneArg{ctx, e.id}));
  return DOTPE_OK;
}

// The scratch goes back at once; the inputs stay with the event until it is
// released (dotpe_lnl_blocks recomputes blocks from them).
static int event_free(Event &e, EventRun &R, cudaStream_t st) {
  (void)e;
  CUDA_OR_FAIL(cudaFreeAsync(R.scr, st));
  R.scr = nullptr;
  return DOTPE_OK;
}

static int autotune_band(dotpe_ctx *ctx, Event &e, EventRun &R, cudaStream_t st);

// The event's cross terms: a cached entry of its bank for its PSD, or a new
// entry computed now for every bank row on `st` (outside any capture) when the
// slice covers at least a quarter of the bank (a smaller slice computes its own
// rows into its scratch instead).  The stream waits for the entry's records.
// Entries past XCACHE_MAX per bank are dropped least recently used first, when
// no event holds them.
static XEntry *xcache_find(Bank &b, uint64_t key, int D) {
  for (XEntry *c : b.xcache)
    if (c->key == key && c->D == D) return c;
  return nullptr;
}

// A new cache entry of the bank's row records for one PSD, computed on `st`
// from omega (which `st` has already been ordered after); evicts the least
// recently used unreferenced entry when the bank's cache is full.
static int xcache_build(dotpe_ctx *ctx, Bank &b, uint64_t key, int D, const float *omega, const double2 *rb_hh,
                        cudaStream_t st, XEntry **out) {
  if ((int)b.xcache.size() >= XCACHE_MAX) {
    auto victim = b.xcache.end();
    for (auto it = b.xcache.begin(); it != b.xcache.end(); ++it)
      if ((*it)->refs == 0 && (victim == b.xcache.end() || (*it)->last < (*victim)->last)) victim = it;
    if (victim != b.xcache.end()) {
      XEntry *v = *victim;
      CUDA_OR_FAIL(cudaEventSynchronize(v->ready));
      CUDA_OR_FAIL(cudaFree(v->mx));
      cudaEventDestroy(v->ready);
      ctx->used -= v->bytes;
      delete v;
      b.xcache.erase(victim);
    }
  }
  XEntry *x = new XEntry();
  x->key = key;
  x->D = D;
  const int rec = (b.n_pol == 2) ? REC_P : REC;
  x->bytes = (size_t)b.I * D * rec * sizeof(float);
  if (cudaMallocAsync((void **)&x->mx, x->bytes, st) != cudaSuccess) {
    cudaGetLastError();
    delete x;
    return fail(DOTPE_E_NOMEM, "cross-term records (%zu bytes)", (size_t)b.I * D * rec * sizeof(float));
  }
  CUDA_OR_FAIL(cudaEventCreateWithFlags(&x->ready, cudaEventDisableTiming));
  if (b.n_pol == 2)
    launch_cross_terms_pol(b.I, 0, b.I, b.M, D, b.B, b.Kpad, b.mode_m, b.master, omega, rb_hh, x->mx, ctx->n_sms,
                           st);
  else
    launch_cross_terms(b.I, 0, b.I, b.M, D, b.B, b.Kpad, b.master, omega, rb_hh, x->mx, ctx->n_sms, st);
  CUDA_OR_FAIL(cudaEventRecord(x->ready, st));
  ctx->used += x->bytes;
  b.xcache.push_back(x);
  *out = x;
  return DOTPE_OK;
}

static int xterms_acquire(dotpe_ctx *ctx, Event &e, EventRun &R, cudaStream_t st) {
  Bank &b = *e.bank;
  XEntry *x = xcache_find(b, e.psd_key, e.D);
  if (x) {
    CUDA_OR_FAIL(cudaStreamWaitEvent(st, x->ready, 0));
  } else if (4 * e.NI < b.I) {
    return DOTPE_OK;
  } else {
    // omega of this event (its prep on `st` writes it) -> records of every bank row
    launch_prep(R.pa, st);
    int rc = xcache_build(ctx, b, e.psd_key, e.D, R.pa.omega, e.rb_hh, st, &x);
    if (rc != DOTPE_OK) return rc;
  }
  x->refs++;
  x->last = now_ns();
  e.xent = x;
  return DOTPE_OK;
}

// Cross-term cache key: FNV-1a over n_det and the PSD bytes (host or device),
// or, with relative binning, over a tag, n_det and the <h|h> weights (complex
// [D][M][M][B]: n = 2 D M M B doubles), which then replace the PSD.
static int psd_hash(int D, int B, const double *psd, uint64_t *out, const double *rb_hh = nullptr, size_t n_rb = 0) {
  const bool rb = rb_hh != nullptr;
  const double *src = rb ? rb_hh : psd;
  std::vector<double> ps(rb ? n_rb : (size_t)D * B);
  if (is_device_ptr(src)) {
    if (cudaMemcpy(ps.data(), src, ps.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(DOTPE_E_DEVICE, "reading the PSD or weights");
  } else {
    memcpy(ps.data(), src, ps.size() * 8);
  }
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](const void *p, size_t n) {
    const uint8_t *c = (const uint8_t *)p;
    for (size_t k = 0; k < n; ++k) h = (h ^ c[k]) * 1099511628211ull;
  };
  if (rb) mix("relative binning", 16);
  mix(&D, sizeof(D));
  mix(ps.data(), ps.size() * 8);
  *out = h;
  return DOTPE_OK;
}

// One event on its slot stream, its slice in bank blocks.
static int run_event(dotpe_ctx *ctx, Event &e) {
  NvtxRange nv("dotpe:event");
  cudaStream_t st = ctx->streams[e.slot];
  EventRun R;
  int rc = event_alloc(ctx, e, st, R);
  if (rc != DOTPE_OK) return rc;
  {
    NvtxRange np("dotpe:prep");
    if ((rc = xterms_acquire(ctx, e, R, st)) != DOTPE_OK) return rc;
    if ((rc = event_begin(e, R, st)) != DOTPE_OK) return rc;
  }
  const int64_t BR = R.L.block_rows;
  const int n_blocks = (int)((e.NI + BR - 1) / BR);
  for (int k = 0; k < n_blocks; ++k) {
    const int64_t r0 = (int64_t)k * BR;
    event_block(ctx, e, R, r0, std::min<int64_t>(BR, e.NI - r0), st);
    if (k == 0 && ctx->autotune && (rc = autotune_band(ctx, e, R, st)) != DOTPE_OK) return rc;
    if (k == 0) CUDA_OR_FAIL(record(e.ev_k0, st));
    {
      NvtxRange nf("dotpe:fused");
      if ((rc = event_fused(ctx, e, R, k == n_blocks - 1, st)) != DOTPE_OK) return rc;
    }
    if (k == n_blocks - 1) CUDA_OR_FAIL(record(e.ev_k1, st));
    R.ra.first = (k == 0);
    NvtxRange nr("dotpe:reduce");
    launch_reduce_block(R.ra, st);
  }
  if ((rc = event_end(ctx, e, R, st)) != DOTPE_OK) return rc;
  return event_free(e, R, st);
}

// ---------------------------------------------------------------------------
// Tile-shape autotuner.  The fused kernel walks the extrinsic tiles in bands:
// every bank tile meets the band's extrinsic tiles before the next band starts,
// so the band's operand stays in L2 while the bank streams once per band.  The
// best band width depends on the operand sizes and on how the two L2 partitions
// share lines, the best tile width (32 samples with two TMEM accumulator sets,
// or 64 with one) on how much the epilogue costs against the MMAs, and whether
// 64-sample tiles run on CTA pairs (cta_group::2, M = 256: each SM loads half
// of the tile's extrinsic rows) or on one SM each on how the mainloop's
// shared-memory ingress weighs against the pair's tail; all three are chosen
// per shape (precision class, modes, k-blocks, extrinsic tiles) by timing
// candidates on the first event of that shape.
// ---------------------------------------------------------------------------
static std::string band_key(const Event &e, const ScratchLayout &L, bool split) {
  char buf[96];
  snprintf(buf, sizeof(buf), "%d/%d/%d/%d/%d", prec_bf16(e.prec) ? 1 : 0, split ? 1 : 0, e.bank->M, e.bank->Kpad,
           L.n_etile);
  return buf;
}

static int event_band(dotpe_ctx *ctx, const Event &e, const ScratchLayout &L, bool split) {
  auto it = ctx->band_cache.find(band_key(e, L, split));
  if (it != ctx->band_cache.end()) return std::min(it->second, L.n_etile);
  return tc_band(ctx->l2_band_bytes, e.bank->Kpad / 64, e.bank->M, split, L.n_etile);
}

// Times the event's first fused launch at candidate (tile form, band width)
// pairs (the event's own inputs, prepared on `st`): 32-sample tiles, and where
// the launch may take them 64-sample tiles on one SM each and on CTA pairs
// (unless the context keeps one SM per tile), band widths doubling from one
// extrinsic tile to all of them.  The results of these runs are overwritten by the real
// launch that follows.  Blocks the calling thread once per shape.
static int autotune_band(dotpe_ctx *ctx, Event &e, EventRun &R, cudaStream_t st) {
  const bool split_main = prec_split(e.prec) && e.prec != DOTPE_PREC_MIXED;
  const std::string key = band_key(e, R.L, prec_split(e.prec));
  if (e.prec == DOTPE_PREC_FP32 || ctx->band_cache.count(key)) return DOTPE_OK;
  TcLaunch T;
  int rc = tc_launch_of(ctx, *e.bank, e.prec, T);
  if (rc != DOTPE_OK) return rc;
  T.split = split_main;
  T.sep = split_main;
  TcWork W = R.W;
  W.P = R.mixed ? screen_params(R) : R.P;
  std::vector<int> tevs{32};
  if (ctx->wide_tiles && !split_main && e.bank->n_pol != 2 && !W.P.lnl_tile && (W.P.gemm_only || W.P.screen_ml))
    tevs.push_back(64);
  // the 64-sample candidates timed as they run: with the <h|h> bound where the event has it
  if (R.mixed && tevs.back() == 64 && (rc = hh_bound_pass(ctx, e, R, W.P, st)) != DOTPE_OK) return rc;
  const int dflt = tc_band(ctx->l2_band_bytes, e.bank->Kpad / 64, e.bank->M, prec_split(e.prec), R.L.n_etile);
  struct Cand { int tev; bool pair; int band; };
  std::vector<Cand> cand;
  for (int tv : tevs) {
    std::vector<int> bands;
    for (int c = 1; c < R.W.n_etile; c *= 2) bands.push_back(c);
    bands.push_back(R.W.n_etile);
    if (std::find(bands.begin(), bands.end(), dflt) == bands.end()) bands.push_back(dflt);
    std::vector<bool> forms{false};
    if (tv == 64 && ctx->pair_tiles) forms.push_back(true);
    for (bool pr : forms)
      for (int c : bands) cand.push_back({tv, pr, c});
  }
  std::vector<cudaEvent_t> ev(cand.size() + 1);
  for (auto &x : ev) CUDA_OR_FAIL(cudaEventCreate(&x));
  // warm-up at the default width, then one timed launch per candidate
  W.band = dflt;
  T.tev = tevs.back();
  T.pair = ctx->pair_tiles;
  int r = launch_tc(T, &W, 1, nullptr, nullptr, st);
  CUDA_OR_FAIL(cudaEventRecord(ev[0], st));
  for (size_t c = 0; c < cand.size() && r == 0; ++c) {
    W.band = cand[c].band;
    T.tev = cand[c].tev;
    T.pair = cand[c].pair;
    r = launch_tc(T, &W, 1, nullptr, nullptr, st);
    CUDA_OR_FAIL(cudaEventRecord(ev[c + 1], st));
  }
  if (r != 0) return fail(DOTPE_E_DEVICE, "autotune launch failed: %s", cudaGetErrorString((cudaError_t)r));
  CUDA_OR_FAIL(cudaEventSynchronize(ev.back()));
  Cand best{tevs.back(), ctx->pair_tiles && tevs.back() == 64, dflt};
  float best_ms = 1e30f;
  for (size_t c = 0; c < cand.size(); ++c) {
    float ms = 0.f;
    CUDA_OR_FAIL(cudaEventElapsedTime(&ms, ev[c], ev[c + 1]));
    if (ms < best_ms) { best_ms = ms; best = cand[c]; }
  }
  for (auto &x : ev) cudaEventDestroy(x);
  ctx->band_cache[key] = best.band;
  ctx->tev_cache[key] = best.tev;
  ctx->pair_cache[key] = best.pair;
  R.W.band = best.band;
  // the tuning runs raised the running maximum and the counters: start the real launch afresh
  CUDA_OR_FAIL(cudaMemsetAsync(R.scr + R.L.ml_running, 0, 4, st));
  CUDA_OR_FAIL(cudaMemsetAsync(R.scr + R.L.n_cand, 0, 16, st));
  return DOTPE_OK;
}

// ---------------------------------------------------------------------------
// A batch of events over one bank in one launch sequence: every event's prep,
// then one persistent fused launch per TC_MAXB events (mixed: screen, one
// selection over the batch, refinement), then every event's reduction.  With
// graphs on, the sequence is captured once per launch and replayed through a
// per-slot executable graph updated in place when the topology repeats.
// ---------------------------------------------------------------------------
static int run_batch(dotpe_ctx *ctx, const std::vector<Event *> &evs, int slot) {
  NvtxRange nv("dotpe:batch");
  cudaStream_t st = ctx->streams[slot];
  const int n = (int)evs.size();
  std::vector<EventRun> R(n);
  for (int k = 0; k < n; ++k) {
    int rc = event_alloc(ctx, *evs[k], st, R[k]);
    if (rc != DOTPE_OK) return rc;
    if ((rc = xterms_acquire(ctx, *evs[k], R[k], st)) != DOTPE_OK) return rc;
  }
  const int prec = evs[0]->prec;
  const bool mixed = (prec == DOTPE_PREC_MIXED);
  int total_tiles = 0;
  for (int k = 0; k < n; ++k) total_tiles += (int)((evs[k]->NI + TC_TI - 1) / TC_TI) * R[k].L.n_etile;
  // batch-wide (event, tile) list of the refinement
  uint8_t *blist = nullptr;
  size_t o_list = 0, o_n = 0, o_counts = 0, o_sep = 0;
  if (mixed) {
    Carver c;
    o_list = c.take<int2>(total_tiles);
    o_n = c.take<int>(1);
    o_counts = c.take<int>(select_count_blocks(total_tiles));
    o_sep = c.take<int>(TC_MAXB);
    CUDA_OR_FAIL(cudaMallocAsync((void **)&blist, c.off, st));
  }
  TcLaunch T;
  if (prec != DOTPE_PREC_FP32) {
    int rc = tc_launch_of(ctx, *evs[0]->bank, prec, T);
    if (rc != DOTPE_OK) return rc;
  }
  const bool capture = ctx->use_graphs;
  if (capture) CUDA_OR_FAIL(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  int rc = DOTPE_OK;
  auto body = [&]() -> int {
    for (int k = 0; k < n; ++k) {
      int r = event_begin(*evs[k], R[k], st);
      if (r != DOTPE_OK) return r;
      event_block(ctx, *evs[k], R[k], 0, evs[k]->NI, st);
      CUDA_OR_FAIL(record(evs[k]->ev_k0, st));
    }
    if (prec == DOTPE_PREC_FP32) {
      for (int k = 0; k < n; ++k) {
        int r = event_fused(ctx, *evs[k], R[k], true, st);
        if (r != DOTPE_OK) return r;
      }
    } else {
      std::vector<TcWork> W(n);
      for (int k0 = 0; k0 < n; k0 += TC_MAXB) {
        const int m = std::min(TC_MAXB, n - k0);
        for (int k = k0; k < k0 + m; ++k) {
          W[k] = R[k].W;
          W[k].P = mixed ? screen_params(R[k]) : R[k].P;
        }
        TcLaunch T1 = T;
        T1.split = prec_split(prec) && !mixed;
        T1.sep = T1.split;
        // one tile width for the launch: 64 samples only if every event takes it
        T1.tev = 64;
        for (int k = k0; k < k0 + m; ++k)
          T1.tev = std::min(T1.tev, launch_tev(ctx, *evs[k], R[k].L, W[k].P, T1.split));
        if (mixed && T1.tev == 64)
          for (int k = k0; k < k0 + m; ++k) {
            int rb = hh_bound_pass(ctx, *evs[k], R[k], W[k].P, st);
            if (rb != DOTPE_OK) return rb;
          }
        int r = launch_tc(T1, &W[k0], m, nullptr, nullptr, st);
        if (r != 0) return fail(DOTPE_E_DEVICE, "tcgen05 batch launch failed: %s", cudaGetErrorString((cudaError_t)r));
      }
      if (mixed) {
        for (int k = 0; k < n; ++k) CUDA_OR_FAIL(record(evs[k]->ev_ks, st));
        int2 *glist = (int2 *)(blist + o_list);
        int *gn = (int *)(blist + o_n);
        for (int k0 = 0; k0 < n; k0 += TC_MAXB) {
          const int m = std::min(TC_MAXB, n - k0);
          SelectBatch sb;
          memset(&sb, 0, sizeof(sb));
          int b0 = 0;
          for (int k = 0; k < m; ++k) {
            sb.ev[k] = select_event_of(R[k0 + k]);
            sb.begin[k] = b0;
            b0 += R[k0 + k].W.n_itile * R[k0 + k].W.n_etile;
          }
          sb.begin[m] = b0;
          sb.n = m;
          sb.list = glist;
          sb.n_list = gn;
          sb.counts = (int *)(blist + o_counts);
          sb.sep = (int *)(blist + o_sep);
          launch_select(sb, st);
          CUDA_OR_FAIL(cudaGetLastError());
          for (int k = k0; k < k0 + m; ++k) W[k].P = refine_params(R[k]);
          TcLaunch T2 = T;
          T2.split = true;
          T2.gate = sb.sep;
          for (int want = 0; want < 2; ++want) {
            T2.sep = want == 1;
            T2.gate_want = want;
            int r = launch_tc(T2, &W[k0], m, glist, gn, st);
            if (r != 0)
              return fail(DOTPE_E_DEVICE, "tcgen05 batch launch failed: %s", cudaGetErrorString((cudaError_t)r));
          }
        }
      }
    }
    for (int k = 0; k < n; ++k) {
      CUDA_OR_FAIL(record(evs[k]->ev_k1, st));
      R[k].ra.first = 1;
      launch_reduce_block(R[k].ra, st);
      int r = event_end(ctx, *evs[k], R[k], st);
      if (r != DOTPE_OK) return r;
    }
    return DOTPE_OK;
  };
  rc = body();
  if (capture) {
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(st, &g);
    if (rc != DOTPE_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (ce != cudaSuccess) return fail(DOTPE_E_DEVICE, "graph capture: %s", cudaGetErrorString(ce));
    char key[64];
    snprintf(key, sizeof(key), "%d/%d", n, prec);
    auto &cache = ctx->graphs[slot];
    auto it = cache.find(key);
    bool ok = false;
    if (it != cache.end()) {
      cudaGraphExecUpdateResultInfo info;
      ok = cudaGraphExecUpdate(it->second, g, &info) == cudaSuccess;
      if (!ok) {
        cudaGetLastError();
        cudaGraphExecDestroy(it->second);
        cache.erase(it);
      }
    }
    if (!ok) {
      cudaGraphExec_t x = nullptr;
      cudaError_t ie = cudaGraphInstantiate(&x, g, 0);
      if (ie != cudaSuccess) {
        cudaGraphDestroy(g);
        return fail(DOTPE_E_DEVICE, "graph instantiate: %s", cudaGetErrorString(ie));
      }
      cache[key] = x;
    }
    cudaError_t le = cudaGraphLaunch(cache[key], st);
    cudaGraphDestroy(g);
    if (le != cudaSuccess) return fail(DOTPE_E_DEVICE, "graph launch: %s", cudaGetErrorString(le));
  } else if (rc != DOTPE_OK) {
    return rc;
  }
  for (int k = 0; k < n; ++k) {
    int r = event_free(*evs[k], R[k], st);
    if (r != DOTPE_OK) return r;
  }
  if (blist) CUDA_OR_FAIL(cudaFreeAsync(blist, st));
  return DOTPE_OK;
}

// Admits queued events in order while a slot and budget are available.
static void progress(dotpe_ctx *ctx) {
  // retire finished events: free their slot and scratch budget
  for (auto &kv : ctx->events) {
    Event &e = *kv.second;
    if (e.state == DOTPE_STATE_RUNNING) {
      cudaError_t q = cudaEventQuery(e.ev_end);
      if (q == cudaSuccess) {
        e.state = (e.h_out->status == 0) ? DOTPE_STATE_DONE : DOTPE_STATE_FAILED;
        {
          std::lock_guard<std::mutex> lk(ctx->cb_mu);
          auto d = ctx->done_ns.find(e.id);
          if (d != ctx->done_ns.end()) {
            e.t_done = d->second;
            ctx->done_ns.erase(d);
          }
        }
        float ms = -1.f;
        if (cudaEventElapsedTime(&ms, e.ev_start, e.ev_end) == cudaSuccess) e.device_ms = ms;
        if (cudaEventElapsedTime(&ms, e.ev_start, e.ev_k0) == cudaSuccess) e.prep_ms = ms;
        if (cudaEventElapsedTime(&ms, e.ev_k0, e.ev_k1) == cudaSuccess) e.fused_ms = ms;
        if (e.prec == DOTPE_PREC_MIXED && cudaEventElapsedTime(&ms, e.ev_ks, e.ev_k1) == cudaSuccess) e.refine_ms = ms;
        if (e.t_done == 0) e.t_done = now_ns();
        ctx->slot_busy[e.slot]--;
        if (e.xent) {
          e.xent->refs--;
          e.xent = nullptr;
        }
        ctx->used = (ctx->used >= e.scratch_bytes) ? ctx->used - e.scratch_bytes : 0;
        e.scratch_bytes = 0;
        if (e.in_stage) {
          cudaFreeHost(e.in_stage);
          e.in_stage = nullptr;
        }
      } else if (q != cudaErrorNotReady) {
        cudaGetLastError();
        e.state = DOTPE_STATE_FAILED;
        ctx->slot_busy[e.slot]--;
      }
    }
  }
  while (!ctx->queue.empty()) {
    uint64_t id = ctx->queue.front();
    auto it = ctx->events.find(id);
    if (it == ctx->events.end()) {
      ctx->queue.pop_front();
      continue;
    }
    Event &e = *it->second;
    int slot = -1;
    for (size_t s = 0; s < ctx->slot_busy.size(); ++s)
      if (!ctx->slot_busy[s]) {
        slot = (int)s;
        break;
      }
    if (slot < 0) break;
    // the launch unit: a submitted batch, or (continuous batching) the queued
    // events of the same bank and precision behind the head, as far as they fit
    std::vector<Event *> grp{&e};
    size_t need = scratch_layout(e).total + keep_bytes_of(e);
    auto batchable = [&](const Event &x) {
      return x.group == 0 && x.bank == e.bank && x.prec == e.prec && x.block_rows == 0 &&
             !(x.flags & DOTPE_FLAG_TEST_STALL) && x.bank->n_pol == 1;
    };
    if (e.group != 0) {
      for (size_t q = 1; q < ctx->queue.size(); ++q) {
        auto jt = ctx->events.find(ctx->queue[q]);
        if (jt == ctx->events.end() || jt->second->group != e.group) break;
        grp.push_back(jt->second);
        need += scratch_layout(*jt->second).total + keep_bytes_of(*jt->second);
      }
    } else if (ctx->max_batch > 1 && batchable(e)) {
      for (size_t q = 1; q < ctx->queue.size() && (int)grp.size() < ctx->max_batch; ++q) {
        auto jt = ctx->events.find(ctx->queue[q]);
        if (jt == ctx->events.end() || !batchable(*jt->second)) break;
        const size_t more = scratch_layout(*jt->second).total + keep_bytes_of(*jt->second);
        if (ctx->used + need + more > ctx->budget) break;
        grp.push_back(jt->second);
        need += more;
      }
    }
    if (ctx->used + need > ctx->budget) break;
    // the screens read the <h|h> bound from the events' own scratch when, for
    // the whole launch unit, that fits too
    for (Event *x : grp) x->want_hb = false;
    if (ctx->wide_tiles) {
      size_t with = 0;
      for (Event *x : grp) with += scratch_layout(*x, true).total + keep_bytes_of(*x);
      if (with > need && ctx->used + with <= ctx->budget) {
        need = with;
        for (Event *x : grp) x->want_hb = true;
      }
    }
    for (size_t q = 0; q < grp.size(); ++q) ctx->queue.pop_front();
    ctx->used += need;
    const int64_t t_admit = now_ns();
    for (Event *x : grp) {
      x->slot = slot;
      x->t_admit = t_admit;
      x->state = DOTPE_STATE_RUNNING;
    }
    ctx->slot_busy[slot] = (int)grp.size();
    const int rc = (grp.size() == 1 && e.group == 0) ? run_event(ctx, e) : run_batch(ctx, grp, slot);
    if (rc != DOTPE_OK) {
      for (Event *x : grp) {
        x->state = DOTPE_STATE_FAILED;
        x->launch_error = g_last_error;
      }
      ctx->slot_busy[slot] = 0;
    }
  }
}

static void free_event(dotpe_ctx *ctx, Event *e) {
  if (e->state == DOTPE_STATE_RUNNING) cudaEventSynchronize(e->ev_end);
  if (e->xent) e->xent->refs--;
  if (e->keep_block) cudaFree(e->keep_block);
  if (e->in_block && e->owns_inputs) cudaFree(e->in_block);
  if (e->in_stage) cudaFreeHost(e->in_stage);
  if (e->h_out) cudaFreeHost(e->h_out);
  if (e->ev_inputs) cudaEventDestroy(e->ev_inputs);
  if (e->ev_start) cudaEventDestroy(e->ev_start);
  if (e->ev_end) cudaEventDestroy(e->ev_end);
  if (e->ev_k0) cudaEventDestroy(e->ev_k0);
  if (e->ev_k1) cudaEventDestroy(e->ev_k1);
  if (e->ev_ks) cudaEventDestroy(e->ev_ks);
  size_t give = e->keep_bytes + e->scratch_bytes + e->in_bytes;
  if (e->state == DOTPE_STATE_QUEUED) give = e->in_bytes;
  ctx->used = (ctx->used >= give) ? ctx->used - give : 0;
  if (e->slot >= 0 && e->state == DOTPE_STATE_RUNNING) ctx->slot_busy[e->slot]--;
  if (e->bank) e->bank->refs--;
  delete e;
}

// ---------------------------------------------------------------------------
// Incoherent single-detector pre-selection (Sec. IV.D, App. B)
// ---------------------------------------------------------------------------
static int preselect_locked(dotpe_ctx *ctx, const dotpe_presel_desc *d, float *lnl_ml, int32_t *arg_ot,
                            double *lnl_inco, int64_t *selected, dotpe_presel_out *out) {
  NvtxRange nv("dotpe:preselect");
  auto bit = ctx->banks.find(d->bank_id);
  if (bit == ctx->banks.end()) return fail(DOTPE_E_NOT_FOUND, "bank %llu", (unsigned long long)d->bank_id);
  Bank &b = *bit->second;
  const bool polb = (b.n_pol == 2);  // polarisation-resolved bank: its own h_imp
  if (!polb && !b.pol) return fail(DOTPE_E_INVALID, "bank %llu was loaded without polarisation factors (pol)",
                                   (unsigned long long)d->bank_id);
  if (d->i0 < 0 || d->i1 <= d->i0 || d->i1 > b.I)
    return fail(DOTPE_E_INVALID, "slice [%lld,%lld) of %lld rows", (long long)d->i0, (long long)d->i1, (long long)b.I);
  if (d->n_det < 1 || d->n_det > MAXD) return fail(DOTPE_E_INVALID, "n_det=%d not in 1..%d", d->n_det, MAXD);
  if (d->n_t < 1 || d->n_t > 4096) return fail(DOTPE_E_INVALID, "n_t=%d not in 1..4096", d->n_t);
  if (d->n_phi < 1 || d->n_phi > PS_MAXPHI) return fail(DOTPE_E_INVALID, "n_phi=%d not in 1..%d", d->n_phi, PS_MAXPHI);
  if (!(d->delta >= 0.0) || !std::isfinite(d->delta)) return fail(DOTPE_E_INVALID, "delta must be finite and >= 0");
  const bool rb = d->rb_dh || d->rb_hh;
  if (rb && !(d->rb_dh && d->rb_hh)) return fail(DOTPE_E_INVALID, "rb_dh and rb_hh go together");
  if ((!rb && (!d->psd || !d->data)) || !d->t_grid) return fail(DOTPE_E_INVALID, "null input array");
  const int prec = d->precision;
  if (polb && rb && prec != DOTPE_PREC_FP32)
    return fail(DOTPE_E_UNSUPPORTED, "pre-selection of a polarisation-resolved bank with relative binning runs in FP32");
  // a polarisation-resolved bank also runs in FP32 (CUDA cores); the tensor-core precisions serve both
  const bool simt_pol = polb && prec == DOTPE_PREC_FP32;
  if (!simt_pol && prec != DOTPE_PREC_FP16 && prec != DOTPE_PREC_FP16X3 && prec != DOTPE_PREC_BF16 &&
      prec != DOTPE_PREC_BF16X3)
    return fail(DOTPE_E_INVALID, "pre-selection precision %d (FP16, FP16X3, BF16 or BF16X3%s)", prec,
                polb ? ", or FP32" : "");
  if (d->flags != 0) return fail(DOTPE_E_INVALID, "flags must be 0");
  const int64_t NI = d->i1 - d->i0;
  if (NI >= (1ll << 31) / 2) return fail(DOTPE_E_UNSUPPORTED, "slice too large");
  const int D = d->n_det, B = b.B, M = b.M, NT = d->n_t;
  const int NTP = (NT + PS_TC - 1) / PS_TC * PS_TC;
  const bool bf = prec_bf16(prec), split = prec_split(prec);
  const int planes = split ? 2 : 1;
  const int J = M * (polb ? 2 : 1);  // data-weight components: (mode, polarisation) pairs j = 2m + p
  const int MG = rb ? J : 1;          // time-grid operands: one per component with relative binning
  cudaStream_t st = ctx->main_stream;

  // cross-term records: the bank's cache entry for this PSD, a new one when the
  // slice is a large part of the bank, else the slice's own
  uint64_t key = 0;
  int rc = rb ? psd_hash(D, B, nullptr, &key, d->rb_hh, (size_t)2 * D * J * J * B) : psd_hash(D, B, d->psd, &key);
  if (rc != DOTPE_OK) return rc;
  XEntry *x = xcache_find(b, key, D);
  const bool build_cache = !x && 4 * NI >= b.I;
  const bool own_mx = !x && !build_cache;

  Carver c;
  const size_t o_psd = c.take<double>((size_t)D * B), o_data = c.take<double2>((size_t)D * B);
  const size_t o_tg = c.take<double>((size_t)D * NT);
  const size_t o_rbd = c.take<double2>(rb ? (size_t)D * J * B : 0), o_rbh = c.take<double2>(rb ? (size_t)D * J * J * B : 0);
  const size_t o_c = c.take<float2>((size_t)D * J * B), o_om = c.take<float>((size_t)D * B);
  const size_t o_fh = c.take<float>(B), o_fl = c.take<float>(B);
  const size_t o_G = c.take<float2>((size_t)MG * D * NTP * B);
  const size_t o_gmax = c.take<float>(1), o_gs = c.take<float>(1);
  const int rec = polb ? REC_P : REC;
  // operand rows per plane: (column, re/im) per mode group, or (column, polarisation, re/im)
  const int64_t g_rows = polb ? (int64_t)4 * D * NTP : (int64_t)MG * 2 * D * NTP;
  const size_t o_Gp = c.take<float2>((polb && !simt_pol) ? (size_t)4 * D * NTP * B : 0);
  const size_t o_GT = c.take<float2>(simt_pol ? (size_t)MG * D * NTP * B : 0);  // the FP32 kernel's layout
  const size_t o_pack = c.take<uint16_t>(simt_pol ? 0 : (size_t)planes * g_rows * b.Kpad);
  const size_t o_mx = own_mx ? c.take<float>((size_t)NI * D * rec) : 0;
  const size_t o_keys = c.take<unsigned long long>((size_t)NI * D);
  const size_t o_ml = c.take<float>((size_t)NI * D), o_arg = c.take<int>((size_t)NI * D * 2);
  const size_t o_inco = c.take<double>(NI), o_sel = c.take<int64_t>(NI);
  const size_t o_maxb = c.take<unsigned long long>(1), o_out = c.take<PreselOut>(1), o_st = c.take<int>(1);
  uint8_t *scr = nullptr;
  if (cudaMallocAsync((void **)&scr, c.off, st) != cudaSuccess) {
    cudaGetLastError();
    return fail(DOTPE_E_NOMEM, "pre-selection scratch (%zu bytes)", c.off);
  }
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  auto finish = [&](int code) {
    cudaStreamSynchronize(st);
    cudaFreeAsync(scr, st);
    cudaStreamSynchronize(st);
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
    return code;
  };
  for (auto &e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) return finish(fail(DOTPE_E_DEVICE, "event creation"));
  auto ck = [&](cudaError_t e, const char *what) {
    if (e != cudaSuccess && rc == DOTPE_OK) rc = fail(DOTPE_E_DEVICE, "%s: %s", what, cudaGetErrorString(e));
  };
  int *status = (int *)(scr + o_st);
  ck(cudaEventRecord(ev[0], st), "event record");
  ck(cudaMemsetAsync(status, 0, sizeof(int), st), "memset");
  ck(cudaMemsetAsync(scr + o_gmax, 0, 4, st), "memset");
  ck(cudaMemsetAsync(scr + o_keys, 0, (size_t)NI * D * 8, st), "memset");
  ck(cudaMemsetAsync(scr + o_maxb, 0, 8, st), "memset");
  if (d->psd) ck(cudaMemcpyAsync(scr + o_psd, d->psd, (size_t)D * B * 8, cudaMemcpyDefault, st), "copying psd");
  if (d->data) ck(cudaMemcpyAsync(scr + o_data, d->data, (size_t)D * B * 16, cudaMemcpyDefault, st), "copying data");
  if (rb) {
    ck(cudaMemcpyAsync(scr + o_rbd, d->rb_dh, (size_t)D * J * B * 16, cudaMemcpyDefault, st), "copying rb_dh");
    ck(cudaMemcpyAsync(scr + o_rbh, d->rb_hh, (size_t)D * J * J * B * 16, cudaMemcpyDefault, st), "copying rb_hh");
  }
  ck(cudaMemcpyAsync(scr + o_tg, d->t_grid, (size_t)D * NT * 8, cudaMemcpyDefault, st), "copying t_grid");
  if (rc != DOTPE_OK) return finish(rc);

  PreselPrepArgs pa;
  memset(&pa, 0, sizeof(pa));
  pa.D = D; pa.B = B; pa.M = rb ? J : M; pa.Kpad = b.Kpad; pa.n_t = NT; pa.n_tpad = NTP;
  pa.rb_dh = rb ? (const double2 *)(scr + o_rbd) : nullptr;
  const double2 *rb_hh = rb ? (const double2 *)(scr + o_rbh) : nullptr;
  pa.f = b.f; pa.w = b.w; pa.psd = (const double *)(scr + o_psd); pa.data = (const double2 *)(scr + o_data);
  pa.t_grid = (const double *)(scr + o_tg);
  pa.c = (float2 *)(scr + o_c); pa.omega = (float *)(scr + o_om);
  pa.fh = (float *)(scr + o_fh); pa.fl = (float *)(scr + o_fl);
  pa.G32 = (float2 *)(scr + o_G); pa.gmax = (float *)(scr + o_gmax);
  pa.gpack = scr + o_pack; pa.pack_kind = polb ? 0 : (bf ? 1 : 2); pa.pack_planes = planes;
  pa.gscale = (float *)(scr + o_gs); pa.status = status;
  launch_presel_prep(pa, st);
  if (simt_pol) launch_transpose_G((int64_t)MG * D, NTP, B, pa.G32, (float2 *)(scr + o_GT), st);
  if (polb && !simt_pol)
    launch_presel_pol_pack((int64_t)D * NTP, B, b.Kpad, pa.G32, (float2 *)(scr + o_Gp), pa.gmax, bf ? 1 : 2, planes,
                           pa.gpack, pa.gscale, st);

  const float *mx = nullptr;
  if (x) {
    ck(cudaStreamWaitEvent(st, x->ready, 0), "cross-term wait");
    mx = x->mx + (size_t)d->i0 * D * rec;
  } else if (build_cache) {
    if ((rc = xcache_build(ctx, b, key, D, pa.omega, rb_hh, st, &x)) != DOTPE_OK) return finish(rc);
    mx = x->mx + (size_t)d->i0 * D * rec;
  } else if (polb) {
    launch_cross_terms_pol(NI, d->i0, b.I, M, D, B, b.Kpad, b.mode_m, b.master, pa.omega, rb_hh,
                           (float *)(scr + o_mx), ctx->n_sms, st);
    mx = (const float *)(scr + o_mx);
  } else {
    launch_cross_terms(NI, d->i0, b.I, M, D, B, b.Kpad, b.master, pa.omega, rb_hh, (float *)(scr + o_mx), ctx->n_sms,
                       st);
    mx = (const float *)(scr + o_mx);
  }
  if (x) {
    x->refs++;
    x->last = now_ns();
  }

  CUtensorMap mapG, mapBank;
  const int64_t a_rows = 2 * (int64_t)M * b.I;
  CUtensorMapDataType dt = bf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  if (simt_pol) {
    // no tensor maps: the FP32 kernel reads the master and the FP32 operand
  } else if (a_rows >= (1ll << 31)) rc = fail(DOTPE_E_UNSUPPORTED, "bank too large for 32-bit TMA coordinates");
  else if (encode_tmap_kblocks(&mapBank, dt, bf ? (void *)b.bf : (void *)b.hf, a_rows, b.Kpad / 64,
                               (uint64_t)b.Kpad * 2, PS_TR, 1) ||
           encode_tmap_kblocks(&mapG, dt, scr + o_pack, (uint64_t)planes * g_rows, b.Kpad / 64,
                               (uint64_t)b.Kpad * 2, 2 * PS_TC, 1))
    rc = fail(DOTPE_E_DEVICE, "cuTensorMapEncodeTiled failed (pre-selection)");
  PreselParams P;
  memset(&P, 0, sizeof(P));
  P.n_rows = (int)NI;
  P.a_row0 = (int)d->i0;
  P.n_det = D; P.n_t = NT; P.n_tpad = NTP; P.n_phi = d->n_phi; P.n_modes = M;
  for (int m = 0; m < MAXM; ++m) P.mode_m[m] = m < M ? b.mode_m[m] : 0;
  {
    int p = 0;
    for (int a = 1; a < MAXM; ++a)
      for (int q = 0; q < a; ++q, ++p) P.pdelta[p] = (a < M) ? (b.mode_m[a] - b.mode_m[q]) : 0;
    // epilogue slots: modes with even m first (the phase pairing phi, phi + pi)
    int ns = 0;
    for (int m = 0; m < M; ++m)
      if (b.mode_m[m] % 2 == 0) P.slot[ns++] = m;
    P.n_even = ns;
    for (int m = 0; m < M; ++m)
      if (b.mode_m[m] % 2 != 0) P.slot[ns++] = m;
    for (; ns < MAXM; ++ns) P.slot[ns] = 0;
    P.slot_mask = (1u << M) - 1u;
    // quarter turns: e^{i m (phi + pi/2)} = i^m e^{i m phi}, so with one mode per
    // class m mod 4 (slot order 0, 2, 1, 3; a mode bank's m are distinct in 1..4)
    // four phases share one rotation; otherwise every phase is rotated on its own
    if (!polb && d->n_phi % 4 == 0) {
      static const int cls_slot[4] = {0, 2, 1, 3};  // class -> slot
      int qs[MAXM] = {0, 0, 0, 0};
      unsigned qm = 0;
      bool ok = true;
      for (int m = 0; m < M && ok; ++m) {
        const int c = ((b.mode_m[m] % 4) + 4) % 4, sl = cls_slot[c];
        if (qm & (1u << sl)) ok = false;
        qm |= 1u << sl;
        qs[sl] = m;
      }
      if (ok) {
        P.quad = 1;
        P.slot_mask = qm;
        for (int q = 0; q < MAXM; ++q) P.slot[q] = qs[q];
      }
    }
  }
  P.n_itile = (int)((NI + PS_TR - 1) / PS_TR);
  P.n_ctile = D * NTP / (polb ? PS_TC / 2 : PS_TC);  // a polarisation-resolved tile holds 32 columns
  P.kb = b.Kpad / 64;
  P.a_plane_rows = M * (int)b.I;
  P.a_mode_rows = (int)b.I;
  P.b_plane_rows = (int)g_rows;
  P.b_mode_rows = rb ? 2 * D * NTP : 0;
  P.pol = b.pol ? b.pol + (size_t)d->i0 * M * 2 : nullptr;
  P.mx = mx;
  P.z_scale = 1.f / (b.a_scale * (bf ? 1.f : FP16_OPERAND_SCALE));
  P.g_scale = pa.gscale;
  P.rank_tol = PS_RANK_TOL;
  P.keys = (unsigned long long *)(scr + o_keys);
  P.status = status;
  P.wait_ns = 4000000000ull;
  if (rc == DOTPE_OK) {
    ck(cudaEventRecord(ev[1], st), "event record");
    if (simt_pol) {
      PreselPolArgs pp;
      memset(&pp, 0, sizeof(pp));
      pp.n_rows = NI; pp.row0 = d->i0; pp.bank_rows = b.I;
      pp.n_det = D; pp.n_t = NT; pp.n_tpad = NTP; pp.n_phi = d->n_phi; pp.n_modes = M; pp.n_bins = B;
      pp.kpad = b.Kpad;
      for (int m = 0; m < MAXM; ++m) pp.mode_m[m] = m < M ? b.mode_m[m] : 0;
      pp.master = b.master;
      pp.G = (const float2 *)(scr + o_GT);
      pp.n_gcomp = MG;
      pp.mx = mx;
      pp.rank_tol = PS_RANK_TOL;
      pp.keys = P.keys;
      launch_presel_pol(pp, st);
      ck(cudaGetLastError(), "pre-selection kernel");
    } else {
      ck((cudaError_t)launch_presel(mapG, mapBank, P, bf, split, rb, polb, ctx->n_sms, st), "pre-selection kernel");
    }
    ck(cudaEventRecord(ev[2], st), "event record");
    launch_presel_finish(NI, D, d->n_phi, d->delta, P.keys, (float *)(scr + o_ml), (int *)(scr + o_arg),
                         (double *)(scr + o_inco), (unsigned long long *)(scr + o_maxb), (int64_t *)(scr + o_sel),
                         (PreselOut *)(scr + o_out), st);
    ck(cudaGetLastError(), "pre-selection finish");
    ck(cudaEventRecord(ev[3], st), "event record");
  }
  PreselOut po;
  int dev_status = 0;
  memset(&po, 0, sizeof(po));
  if (rc == DOTPE_OK) {
    ck(cudaMemcpyAsync(&po, scr + o_out, sizeof(po), cudaMemcpyDeviceToHost, st), "result copy");
    ck(cudaMemcpyAsync(&dev_status, status, sizeof(int), cudaMemcpyDeviceToHost, st), "result copy");
    ck(cudaStreamSynchronize(st), "pre-selection");
  }
  if (x) x->refs--;
  if (rc != DOTPE_OK) return finish(rc);
  if (dev_status != 0) {
    rc = dev_status == DEV_E_TIMEOUT ? fail(DOTPE_E_TIMEOUT, "a device wait ran out in the pre-selection kernel")
                                     : fail(DOTPE_E_INVALID, "non-finite values in the pre-selection inputs");
    return finish(rc);
  }
  if (lnl_ml) ck(cudaMemcpyAsync(lnl_ml, scr + o_ml, (size_t)NI * D * 4, cudaMemcpyDefault, st), "copying lnl_ml");
  if (arg_ot) ck(cudaMemcpyAsync(arg_ot, scr + o_arg, (size_t)NI * D * 8, cudaMemcpyDefault, st), "copying arg_ot");
  if (lnl_inco) ck(cudaMemcpyAsync(lnl_inco, scr + o_inco, (size_t)NI * 8, cudaMemcpyDefault, st), "copying lnl_inco");
  if (selected && po.n_selected > 0)
    ck(cudaMemcpyAsync(selected, scr + o_sel, (size_t)po.n_selected * 8, cudaMemcpyDefault, st), "copying selected");
  ck(cudaStreamSynchronize(st), "pre-selection outputs");
  if (out) {
    memset(out, 0, sizeof(*out));
    out->max_lnl_inco = po.max_inco;
    out->threshold = po.threshold;
    out->arg_i = po.arg_i;
    out->n_selected = po.n_selected;
    cudaEventElapsedTime(&out->kernel_ms, ev[1], ev[2]);
    cudaEventElapsedTime(&out->device_ms, ev[0], ev[3]);
    out->device_status = dev_status;
  }
  return finish(rc);
}

// ---------------------------------------------------------------------------
// Relative-binning weights (App. A)
// ---------------------------------------------------------------------------
static int rb_weights_locked(dotpe_ctx *ctx, const dotpe_rb_desc *d, double *w_dh, double *w_hh) {
  NvtxRange nv("dotpe:rb_weights");
  if (d->n_det < 1 || d->n_det > MAXD) return fail(DOTPE_E_INVALID, "n_det=%d not in 1..%d", d->n_det, MAXD);
  if (d->n_modes < 1 || d->n_modes > 2 * MAXM)
    return fail(DOTPE_E_INVALID, "n_modes=%d components not in 1..%d", d->n_modes, 2 * MAXM);
  if (d->n_bins < 2 || d->n_fine < d->n_bins) return fail(DOTPE_E_INVALID, "n_bins=%d, n_fine=%lld", d->n_bins,
                                                           (long long)d->n_fine);
  if (!d->f_fine || !d->df_fine || !d->psd || !d->data || !d->h0 || !d->nodes || !w_dh || !w_hh)
    return fail(DOTPE_E_INVALID, "null array");
  const int D = d->n_det, M = d->n_modes, B = d->n_bins;
  const int64_t N = d->n_fine;
  std::vector<int64_t> nodes(B);
  if (is_device_ptr(d->nodes)) CUDA_OR_FAIL(cudaMemcpy(nodes.data(), d->nodes, B * 8, cudaMemcpyDeviceToHost));
  else memcpy(nodes.data(), d->nodes, B * 8);
  for (int b = 0; b < B; ++b)
    if (nodes[b] < 0 || nodes[b] >= N || (b > 0 && nodes[b] <= nodes[b - 1]))
      return fail(DOTPE_E_INVALID, "nodes must be strictly increasing indices into f_fine (node %d = %lld)", b,
                  (long long)nodes[b]);
  cudaStream_t st = ctx->main_stream;
  Carver c;
  const size_t o_f = c.take<double>(N), o_df = c.take<double>(N), o_psd = c.take<double>((size_t)D * N);
  const size_t o_data = c.take<double2>((size_t)D * N), o_h0 = c.take<double2>((size_t)M * N);
  const size_t o_t0 = c.take<double>(D), o_nodes = c.take<int64_t>(B);
  const size_t o_wdh = c.take<double2>((size_t)D * M * B), o_whh = c.take<double2>((size_t)D * M * M * B);
  const size_t o_st = c.take<int>(1);
  uint8_t *scr = nullptr;
  if (cudaMallocAsync((void **)&scr, c.off, st) != cudaSuccess) {
    cudaGetLastError();
    return fail(DOTPE_E_NOMEM, "relative-binning scratch (%zu bytes)", c.off);
  }
  int rc = DOTPE_OK;
  auto ck = [&](cudaError_t e, const char *what) {
    if (e != cudaSuccess && rc == DOTPE_OK) rc = fail(DOTPE_E_DEVICE, "%s: %s", what, cudaGetErrorString(e));
  };
  ck(cudaMemsetAsync(scr + o_st, 0, sizeof(int), st), "memset");
  ck(cudaMemsetAsync(scr + o_t0, 0, D * 8, st), "memset");
  ck(cudaMemcpyAsync(scr + o_f, d->f_fine, N * 8, cudaMemcpyDefault, st), "copying f_fine");
  ck(cudaMemcpyAsync(scr + o_df, d->df_fine, N * 8, cudaMemcpyDefault, st), "copying df_fine");
  ck(cudaMemcpyAsync(scr + o_psd, d->psd, (size_t)D * N * 8, cudaMemcpyDefault, st), "copying psd");
  ck(cudaMemcpyAsync(scr + o_data, d->data, (size_t)D * N * 16, cudaMemcpyDefault, st), "copying data");
  ck(cudaMemcpyAsync(scr + o_h0, d->h0, (size_t)M * N * 16, cudaMemcpyDefault, st), "copying h0");
  if (d->t0) ck(cudaMemcpyAsync(scr + o_t0, d->t0, D * 8, cudaMemcpyDefault, st), "copying t0");
  ck(cudaMemcpyAsync(scr + o_nodes, nodes.data(), B * 8, cudaMemcpyHostToDevice, st), "copying nodes");
  if (rc == DOTPE_OK) {
    launch_rb_weights(D, M, N, (const double *)(scr + o_f), (const double *)(scr + o_df),
                      (const double *)(scr + o_psd), (const double2 *)(scr + o_data), (const double2 *)(scr + o_h0),
                      (const double *)(scr + o_t0), B, (const int64_t *)(scr + o_nodes), (double2 *)(scr + o_wdh),
                      (double2 *)(scr + o_whh), (int *)(scr + o_st), st);
    ck(cudaGetLastError(), "relative-binning weights kernel");
  }
  int dev_status = 0;
  if (rc == DOTPE_OK) {
    ck(cudaMemcpyAsync(&dev_status, scr + o_st, sizeof(int), cudaMemcpyDeviceToHost, st), "status copy");
    ck(cudaStreamSynchronize(st), "relative-binning weights");
  }
  if (rc == DOTPE_OK && dev_status != 0)
    rc = fail(DOTPE_E_INVALID, dev_status == DEV_E_SHAPE ? "a reference mode vanishes at a node"
                                                          : "non-finite or non-positive PSD, or non-finite inputs");
  if (rc == DOTPE_OK) {
    ck(cudaMemcpyAsync(w_dh, scr + o_wdh, (size_t)D * M * B * 16, cudaMemcpyDefault, st), "copying w_dh");
    ck(cudaMemcpyAsync(w_hh, scr + o_whh, (size_t)D * M * M * B * 16, cudaMemcpyDefault, st), "copying w_hh");
    ck(cudaStreamSynchronize(st), "relative-binning outputs");
  }
  cudaStreamSynchronize(st);
  cudaFreeAsync(scr, st);
  cudaStreamSynchronize(st);
  return rc;
}

// ---------------------------------------------------------------------------
// Posterior samples (Eq. posterior_element resampling, App. C distance draws)
// ---------------------------------------------------------------------------
static int samples_locked(dotpe_ctx *ctx, Event &e, int64_t n, const double *uniforms, int64_t *i_out,
                          int64_t *e_out, int32_t *o_out, double *d_out) {
  NvtxRange nv("dotpe:posterior_samples");
  Bank &b = *e.bank;
  if (!(e.flags & DOTPE_FLAG_STORE_LNL))
    return fail(DOTPE_E_INVALID, "posterior samples need an event run with DOTPE_FLAG_STORE_LNL");
  if (n < 1 || n > (1ll << 24)) return fail(DOTPE_E_INVALID, "n=%lld not in 1..2^24", (long long)n);
  if (!uniforms) return fail(DOTPE_E_INVALID, "null uniforms");
  cudaStream_t st = ctx->main_stream;
  Carver c;
  const size_t o_u = c.take<double>((size_t)4 * n), o_cdf = c.take<double>(e.NI);
  const size_t o_i = c.take<int64_t>(n), o_e = c.take<int64_t>(n), o_o = c.take<int32_t>(n), o_d = c.take<double>(n);
  const size_t o_st = c.take<int>(1);
  uint8_t *scr = nullptr;
  if (cudaMallocAsync((void **)&scr, c.off, st) != cudaSuccess) {
    cudaGetLastError();
    return fail(DOTPE_E_NOMEM, "sampling scratch (%zu bytes)", c.off);
  }
  int rc = DOTPE_OK;
  auto ck = [&](cudaError_t x, const char *what) {
    if (x != cudaSuccess && rc == DOTPE_OK) rc = fail(DOTPE_E_DEVICE, "%s: %s", what, cudaGetErrorString(x));
  };
  ck(cudaMemsetAsync(scr + o_st, 0, sizeof(int), st), "memset");
  ck(cudaMemcpyAsync(scr + o_u, uniforms, (size_t)32 * n, cudaMemcpyDefault, st), "copying uniforms");
  SampleArgs a;
  memset(&a, 0, sizeof(a));
  a.n_int = e.NI;
  a.n_ext = e.NE;
  a.n_det = e.D;
  a.n_modes = b.M;
  a.n_bins = b.B;
  a.n_phi = e.nphi;
  for (int m = 0; m < MAXM; ++m) a.mode_m[m] = m < b.M ? b.mode_m[m] : 0;
  a.i_base = e.i0;
  a.bank_rows = b.I;
  a.kpad = b.Kpad;
  a.master = b.master;
  a.f = b.f;
  a.w = b.w;
  a.psd = e.psd;
  a.data = e.data;
  a.rb_dh = e.rb_dh;
  a.rb_hh = e.rb_hh;
  a.t = e.t;
  a.R = e.R;
  a.F = e.F;
  a.n_pol = b.n_pol;
  a.lw_ext = e.has_lwe ? e.lwe : nullptr;
  a.ln_p_int = e.ln_p_int;
  a.lnl = e.lnl_tile;
  a.threshold = e.h_out->threshold;
  a.u_min = (float)e.u_min;
  a.dm_table = ctx->dm_table;
  a.status = (int *)(scr + o_st);
  if (rc == DOTPE_OK) {
    launch_sample(a, n, (const double *)(scr + o_u), (double *)(scr + o_cdf), (int64_t *)(scr + o_i),
                  (int64_t *)(scr + o_e), (int32_t *)(scr + o_o), (double *)(scr + o_d), st);
    ck(cudaGetLastError(), "sampling kernels");
  }
  int dev_status = 0;
  if (rc == DOTPE_OK) {
    ck(cudaMemcpyAsync(&dev_status, scr + o_st, sizeof(int), cudaMemcpyDeviceToHost, st), "status copy");
    ck(cudaStreamSynchronize(st), "sampling");
  }
  if (rc == DOTPE_OK && dev_status != 0) rc = fail(DOTPE_E_INVALID, "no pair or phase of positive weight");
  if (rc == DOTPE_OK) {
    if (i_out) ck(cudaMemcpyAsync(i_out, scr + o_i, 8 * n, cudaMemcpyDefault, st), "copying i");
    if (e_out) ck(cudaMemcpyAsync(e_out, scr + o_e, 8 * n, cudaMemcpyDefault, st), "copying e");
    if (o_out) ck(cudaMemcpyAsync(o_out, scr + o_o, 4 * n, cudaMemcpyDefault, st), "copying o");
    if (d_out) ck(cudaMemcpyAsync(d_out, scr + o_d, 8 * n, cudaMemcpyDefault, st), "copying distances");
    ck(cudaStreamSynchronize(st), "sampling outputs");
  }
  cudaStreamSynchronize(st);
  cudaFreeAsync(scr, st);
  cudaStreamSynchronize(st);
  return rc;
}

}  // namespace dotpe

using namespace dotpe;

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char *dotpe_strerror(int s) {
  switch (s) {
    case DOTPE_OK: return "ok";
    case DOTPE_E_INVALID: return "invalid argument";
    case DOTPE_E_NOMEM: return "out of memory";
    case DOTPE_E_ADMISSION: return "event can never fit the HBM budget";
    case DOTPE_E_NOT_READY: return "not ready";
    case DOTPE_E_TIMEOUT: return "timeout";
    case DOTPE_E_DEVICE: return "CUDA device error";
    case DOTPE_E_NOT_FOUND: return "not found";
    case DOTPE_E_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

const char *dotpe_last_error_message(void) { return g_last_error.c_str(); }

int dotpe_version(void) { return DOTPE_ABI_VERSION; }

int dotpe_create(const dotpe_config *cfg, dotpe_ctx **out) {
  if (!out) return fail(DOTPE_E_INVALID, "out is null");
  *out = nullptr;
  dotpe_config c;
  memset(&c, 0, sizeof(c));
  if (cfg) c = *cfg;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    cudaGetLastError();
    return fail(DOTPE_E_DEVICE, "no CUDA device");
  }
  if (c.device < 0 || c.device >= ndev) return fail(DOTPE_E_INVALID, "device %d out of range", c.device);
  CUDA_OR_FAIL(cudaSetDevice(c.device));
  cudaDeviceProp prop;
  CUDA_OR_FAIL(cudaGetDeviceProperties(&prop, c.device));
  if (prop.major < 10) return fail(DOTPE_E_UNSUPPORTED, "device %s (sm_%d%d) lacks tcgen05", prop.name, prop.major, prop.minor);
  dotpe_ctx *ctx = new dotpe_ctx();
  ctx->device = c.device;
  ctx->n_sms = prop.multiProcessorCount;
  snprintf(ctx->name, sizeof(ctx->name), "%s", prop.name);
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  ctx->budget = c.hbm_budget_bytes ? c.hbm_budget_bytes : (uint64_t)(0.9 * (double)fr);
  // a third of L2 for the resident extrinsic band: the rest serves the streaming
  // bank tiles and the two L2 partitions' duplicates
  ctx->l2_band_bytes = prop.l2CacheSize / 3.0;
  if (const char *v = getenv("DOTPE_L2_BAND_MB")) ctx->l2_band_bytes = atof(v) * 1048576.0;

  int ns = c.n_slots > 0 ? c.n_slots : 4;
  ctx->max_batch = c.max_batch > 1 ? c.max_batch : 1;
  ctx->autotune = (c.flags & DOTPE_CONFIG_AUTOTUNE) != 0;
  ctx->wide_tiles = (c.flags & DOTPE_CONFIG_NARROW_TILES) == 0;
  ctx->pair_tiles = (c.flags & DOTPE_CONFIG_SINGLE_CTA_TILES) == 0;
  ctx->use_graphs = (c.flags & DOTPE_CONFIG_NO_GRAPHS) == 0;
  ctx->graphs.resize(ns);
  ctx->streams.resize(ns);
  ctx->slot_busy.assign(ns, 0);
  for (int s = 0; s < ns; ++s) cudaStreamCreateWithFlags(&ctx->streams[s], cudaStreamNonBlocking);
  cudaStreamCreateWithFlags(&ctx->main_stream, cudaStreamNonBlocking);
  cudaStreamCreateWithFlags(&ctx->input_stream, cudaStreamNonBlocking);
  // keep freed stream-ordered memory in the pool for reuse
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, c.device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  {
    char msg[160];
    const int trc = shared_dm_table(c.device, ctx->main_stream, &ctx->dm_table, msg, sizeof(msg));
    if (trc != DOTPE_OK) {
      for (auto s : ctx->streams) cudaStreamDestroy(s);
      cudaStreamDestroy(ctx->main_stream);
      cudaStreamDestroy(ctx->input_stream);
      delete ctx;
      return fail(trc, "%s", msg);
    }
  }
  // admission worker: admits queued events as earlier ones complete
  ctx->worker = std::thread([ctx]() {
    cudaSetDevice(ctx->device);
    while (true) {
      {
        std::unique_lock<std::mutex> lk(ctx->cb_mu);
        ctx->cv.wait_for(lk, std::chrono::milliseconds(2));
        if (ctx->stop) return;
      }
      std::lock_guard<std::mutex> lk(ctx->mu);
      if (!ctx->queue.empty()) progress(ctx);
    }
  });
  *out = ctx;
  return DOTPE_OK;
}

int dotpe_destroy(dotpe_ctx *ctx) {
  if (!ctx) return fail(DOTPE_E_INVALID, "ctx is null");
  {
    std::lock_guard<std::mutex> lk(ctx->cb_mu);
    ctx->stop = true;
  }
  ctx->cv.notify_all();
  if (ctx->worker.joinable()) ctx->worker.join();
  cudaSetDevice(ctx->device);
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    for (auto &kv : ctx->events) free_event(ctx, kv.second);
    ctx->events.clear();
    for (auto &kv : ctx->banks) {
      cudaFree(kv.second->block);
      delete kv.second;
    }
    ctx->banks.clear();
  }
  cudaDeviceSynchronize();
  for (auto &m : ctx->graphs)
    for (auto &kv : m) cudaGraphExecDestroy(kv.second);
  for (auto s : ctx->streams) cudaStreamDestroy(s);
  cudaStreamDestroy(ctx->main_stream);
  cudaStreamDestroy(ctx->input_stream);
  delete ctx;
  return DOTPE_OK;
}

int dotpe_device_info(dotpe_ctx *ctx, int *n_sms, char *name, int name_len) {
  if (!ctx) return fail(DOTPE_E_INVALID, "ctx is null");
  if (n_sms) *n_sms = ctx->n_sms;
  if (name && name_len > 0) snprintf(name, (size_t)name_len, "%s", ctx->name);
  return DOTPE_OK;
}

// copies n bytes from a host or device pointer into device memory
static int copy_in(void *dst, const void *src, size_t n, cudaStream_t st) {
  if (n == 0) return DOTPE_OK;
  CUDA_OR_FAIL(cudaMemcpyAsync(dst, src, n, cudaMemcpyDefault, st));
  return DOTPE_OK;
}

int dotpe_bank_load(dotpe_ctx *ctx, const dotpe_bank_desc *d, uint64_t *bank_id) {
  if (!ctx || !d || !bank_id) return fail(DOTPE_E_INVALID, "null argument");
  if (d->n_int < 1 || d->n_modes < 1 || d->n_modes > MAXM || d->n_bins < 2 || !d->mode_m || !d->f || !d->w_quad ||
      !d->h)
    return fail(DOTPE_E_INVALID, "bank shape: n_int=%lld n_modes=%d n_bins=%d", (long long)d->n_int, d->n_modes,
                d->n_bins);
  if (d->h_dtype != DOTPE_C128 && d->h_dtype != DOTPE_C64) return fail(DOTPE_E_INVALID, "h_dtype");
  if (d->n_pol < 0 || d->n_pol > 2) return fail(DOTPE_E_INVALID, "n_pol=%d not in 0..2", d->n_pol);
  for (int m = 0; m < d->n_modes; ++m) {
    if (d->mode_m[m] < 1 || d->mode_m[m] > 4) return fail(DOTPE_E_INVALID, "mode_m[%d]=%d not in 1..4", m, d->mode_m[m]);
    if (m > 0 && d->mode_m[m] <= d->mode_m[m - 1]) return fail(DOTPE_E_INVALID, "mode_m must increase");
  }
  std::lock_guard<std::mutex> lk(ctx->mu);
  CUDA_OR_FAIL(cudaSetDevice(ctx->device));
  Bank *b = new Bank();
  b->I = d->n_int;
  b->M = d->n_modes;
  b->B = d->n_bins;
  b->n_pol = (d->n_pol == 2) ? 2 : 1;
  b->Kpad = (int)(((2 * b->n_pol * (int64_t)d->n_bins + 63) / 64) * 64);
  for (int m = 0; m < d->n_modes; ++m) b->mode_m[m] = d->mode_m[m];
  const size_t nel = (size_t)b->M * b->I * b->Kpad;
  Carver c;
  size_t o_f = c.take<double>(b->B), o_w = c.take<double>(b->B), o_lw = c.take<double>(b->I);
  size_t o_master = c.take<float>(nel), o_bf = c.take<__nv_bfloat16>(2 * nel), o_hf = c.take<__half>(2 * nel);
  size_t o_scal = c.take<float>(4);
  size_t o_pol = d->pol ? c.take<float2>((size_t)b->I * b->M * 2) : 0;
  b->bytes = c.off;
  if (ctx->used + b->bytes > ctx->budget) {
    delete b;
    return fail(DOTPE_E_NOMEM, "bank needs %zu bytes beyond the budget", c.off);
  }
  cudaError_t e = cudaMalloc(&b->block, b->bytes);
  if (e != cudaSuccess) {
    delete b;
    return fail(DOTPE_E_NOMEM, "bank allocation of %zu bytes: %s", c.off, cudaGetErrorString(e));
  }
  uint8_t *base = (uint8_t *)b->block;
  b->f = (double *)(base + o_f);
  b->w = (double *)(base + o_w);
  b->lw = d->ln_w_int ? (double *)(base + o_lw) : nullptr;
  b->master = (float *)(base + o_master);
  b->bf = (__nv_bfloat16 *)(base + o_bf);
  b->hf = (__half *)(base + o_hf);
  float *scal = (float *)(base + o_scal);  // [0] amax, [1] a_scale, [2] status
  b->pol = d->pol ? (float2 *)(base + o_pol) : nullptr;
  cudaStream_t st = ctx->main_stream;
  int rc = DOTPE_OK;
  auto check = [&](cudaError_t x) {
    if (x != cudaSuccess && rc == DOTPE_OK) rc = fail(DOTPE_E_DEVICE, "bank load: %s", cudaGetErrorString(x));
  };
  check(cudaMemsetAsync(b->master, 0, nel * sizeof(float), st));
  check(cudaMemsetAsync(scal, 0, 16, st));
  check(cudaMemcpyAsync(b->f, d->f, b->B * 8, cudaMemcpyDefault, st));
  check(cudaMemcpyAsync(b->w, d->w_quad, b->B * 8, cudaMemcpyDefault, st));
  if (d->ln_w_int) check(cudaMemcpyAsync(b->lw, d->ln_w_int, b->I * 8, cudaMemcpyDefault, st));
  if (d->pol && rc == DOTPE_OK) {
    // polarisation factors: FP64 complex -> FP32 on the host, then one copy
    const size_t n = (size_t)b->I * b->M * 2;
    std::vector<double> src;
    const double *pd = d->pol;
    if (is_device_ptr(d->pol)) {
      src.resize(2 * n);
      check(cudaMemcpy(src.data(), d->pol, 2 * n * sizeof(double), cudaMemcpyDeviceToHost));
      pd = src.data();
    }
    std::vector<float2> pf(n);
    bool finite = true;
    for (size_t k = 0; k < n && rc == DOTPE_OK; ++k) {
      if (!std::isfinite(pd[2 * k]) || !std::isfinite(pd[2 * k + 1])) finite = false;
      pf[k] = make_float2((float)pd[2 * k], (float)pd[2 * k + 1]);
    }
    if (!finite && rc == DOTPE_OK) rc = fail(DOTPE_E_INVALID, "pol contains non-finite values");
    if (rc == DOTPE_OK) check(cudaMemcpy(b->pol, pf.data(), n * sizeof(float2), cudaMemcpyHostToDevice));
  }
  // stream the waveforms through a device staging buffer in row chunks
  const size_t row_bytes = (size_t)b->M * b->n_pol * b->B * (d->h_dtype == DOTPE_C128 ? 16 : 8);
  const bool hdev = is_device_ptr(d->h);
  int64_t chunk = (int64_t)((256u << 20) / row_bytes);
  if (chunk < 1) chunk = 1;
  void *stage = nullptr;
  void *pin = nullptr;
  if (!hdev) {
    check(cudaMalloc(&stage, (size_t)std::min<int64_t>(chunk, b->I) * row_bytes));
    check(cudaHostAlloc(&pin, (size_t)std::min<int64_t>(chunk, b->I) * row_bytes, cudaHostAllocDefault));
  }
  for (int64_t r0 = 0; r0 < b->I && rc == DOTPE_OK; r0 += chunk) {
    int64_t rows = std::min<int64_t>(chunk, b->I - r0);
    const uint8_t *src = (const uint8_t *)d->h + (size_t)r0 * row_bytes;
    const void *dsrc = src;
    if (!hdev) {
      check(cudaStreamSynchronize(st));  // previous chunk done with the pinned buffer
      memcpy(pin, src, (size_t)rows * row_bytes);
      check(cudaMemcpyAsync(stage, pin, (size_t)rows * row_bytes, cudaMemcpyHostToDevice, st));
      dsrc = stage;
    }
    launch_bank_to_master(rows, r0, b->I, b->M, b->B, b->Kpad, b->n_pol, dsrc, d->h_dtype, b->master, &scal[0],
                          (int *)&scal[2], st);
  }
  launch_master_to_planes((int64_t)nel, b->master, &scal[0], b->bf, b->hf, &scal[1], st);
  check(cudaGetLastError());
  check(cudaStreamSynchronize(st));
  if (stage) cudaFree(stage);
  if (pin) cudaFreeHost(pin);
  float hs[4] = {0, 0, 0, 0};
  if (rc == DOTPE_OK) check(cudaMemcpy(hs, scal, 16, cudaMemcpyDeviceToHost));
  if (rc == DOTPE_OK && *(int *)&hs[2] != 0) rc = fail(DOTPE_E_INVALID, "bank contains non-finite values");
  if (rc == DOTPE_OK && !(hs[0] > 0.f)) rc = fail(DOTPE_E_INVALID, "bank is all zero");
  if (rc != DOTPE_OK) {
    cudaFree(b->block);
    delete b;
    return rc;
  }
  b->a_scale = hs[1];
  b->id = ctx->next_id++;
  ctx->banks[b->id] = b;
  ctx->used += b->bytes;
  *bank_id = b->id;
  return DOTPE_OK;
}

}  // extern "C"

// ---- bank files (checkpoint / resume) ----
// Little-endian, host-native: the header, then the payload f [B], w [B],
// ln w_int [I] (if present), the FP32 master [M][I][Kpad], the polarisation
// factors [I][M][2] float2 (if present); FNV-1a 64 over the header (its
// checksum field zeroed) and then the payload, so a damaged mode number, scale
// or polarisation count is refused like a damaged payload.  The operand planes
// are rebuilt on open at the saved scale, so they equal the saved bank's planes.
struct BankFileHeader {
  char magic[8];
  uint32_t version, n_pol;
  int64_t n_int;
  int32_t n_modes, n_bins, kpad, has_lw, has_pol;
  int32_t mode_m[MAXM];
  float a_scale;
  uint64_t payload_bytes, checksum;
};
static const char BANK_MAGIC[8] = {'D', 'O', 'T', 'P', 'E', 'B', 'K', '1'};
static const uint32_t BANK_VERSION = 2;  // 2: the checksum covers the header

static uint64_t fnv1a(uint64_t h, const uint8_t *p, size_t n) {
  for (size_t k = 0; k < n; ++k) {
    h ^= p[k];
    h *= 1099511628211ull;
  }
  return h;
}
static uint64_t header_hash(const BankFileHeader &h) {
  BankFileHeader z = h;
  z.checksum = 0;
  return fnv1a(1469598103934665603ull, reinterpret_cast<const uint8_t *>(&z), sizeof(z));
}

// One allocation for a bank's arrays (the layout of dotpe_bank_load); pointers set, nothing copied.
static int bank_alloc(dotpe_ctx *ctx, int64_t I, int M, int B, int Kpad, int n_pol, bool has_lw, bool has_pol,
                      size_t extra_bytes, Bank **out, uint8_t **extra) {
  Bank *b = new Bank();
  b->I = I; b->M = M; b->B = B; b->Kpad = Kpad; b->n_pol = n_pol;
  const size_t nel = (size_t)M * I * Kpad;
  Carver c;
  size_t o_f = c.take<double>(B), o_w = c.take<double>(B), o_lw = c.take<double>(has_lw ? I : 0);
  size_t o_master = c.take<float>(nel), o_bf = c.take<__nv_bfloat16>(2 * nel), o_hf = c.take<__half>(2 * nel);
  size_t o_pol = c.take<float2>(has_pol ? (size_t)I * M * 2 : 0);
  size_t o_extra = c.take<uint8_t>(extra_bytes);
  b->bytes = c.off;
  if (ctx->used + b->bytes > ctx->budget) {
    delete b;
    return fail(DOTPE_E_NOMEM, "bank needs %zu bytes beyond the budget", c.off);
  }
  if (cudaMalloc(&b->block, b->bytes) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return fail(DOTPE_E_NOMEM, "bank allocation of %zu bytes", c.off);
  }
  uint8_t *base = (uint8_t *)b->block;
  b->f = (double *)(base + o_f);
  b->w = (double *)(base + o_w);
  b->lw = has_lw ? (double *)(base + o_lw) : nullptr;
  b->master = (float *)(base + o_master);
  b->bf = (__nv_bfloat16 *)(base + o_bf);
  b->hf = (__half *)(base + o_hf);
  b->pol = has_pol ? (float2 *)(base + o_pol) : nullptr;
  if (extra) *extra = base + o_extra;
  *out = b;
  return DOTPE_OK;
}

extern "C" {

int dotpe_bank_save(dotpe_ctx *ctx, uint64_t bank_id, const char *path) {
  if (!ctx || !path) return fail(DOTPE_E_INVALID, "null argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->banks.find(bank_id);
  if (it == ctx->banks.end()) return fail(DOTPE_E_NOT_FOUND, "bank %llu", (unsigned long long)bank_id);
  const Bank &b = *it->second;
  CUDA_OR_FAIL(cudaSetDevice(ctx->device));
  CUDA_OR_FAIL(cudaDeviceSynchronize());
  struct Part { const void *src; size_t n; };
  const Part parts[5] = {{b.f, (size_t)b.B * 8}, {b.w, (size_t)b.B * 8}, {b.lw, b.lw ? (size_t)b.I * 8 : 0},
                         {b.master, (size_t)b.M * b.I * b.Kpad * 4}, {b.pol, b.pol ? (size_t)b.I * b.M * 16 : 0}};
  BankFileHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, BANK_MAGIC, 8);
  h.version = BANK_VERSION;
  h.n_pol = (uint32_t)b.n_pol;
  h.n_int = b.I;
  h.n_modes = b.M; h.n_bins = b.B; h.kpad = b.Kpad;
  h.has_lw = b.lw != nullptr; h.has_pol = b.pol != nullptr;
  for (int m = 0; m < MAXM; ++m) h.mode_m[m] = b.mode_m[m];
  h.a_scale = b.a_scale;
  for (const Part &p : parts) h.payload_bytes += p.n;
  FILE *fp = fopen(path, "wb");
  if (!fp) return fail(DOTPE_E_INVALID, "cannot open %s for writing", path);
  const size_t chunk = (size_t)64 << 20;
  std::vector<uint8_t> buf(chunk);
  uint64_t sum = header_hash(h);
  bool ok = fwrite(&h, sizeof(h), 1, fp) == 1;
  for (const Part &p : parts)
    for (size_t o = 0; ok && o < p.n; o += chunk) {
      const size_t n = std::min(chunk, p.n - o);
      if (cudaMemcpy(buf.data(), (const uint8_t *)p.src + o, n, cudaMemcpyDeviceToHost) != cudaSuccess) {
        fclose(fp);
        return fail(DOTPE_E_DEVICE, "bank save: copy from the device");
      }
      sum = fnv1a(sum, buf.data(), n);
      ok = fwrite(buf.data(), 1, n, fp) == n;
    }
  h.checksum = sum;
  ok = ok && fseek(fp, 0, SEEK_SET) == 0 && fwrite(&h, sizeof(h), 1, fp) == 1;
  ok = (fclose(fp) == 0) && ok;
  return ok ? DOTPE_OK : fail(DOTPE_E_INVALID, "writing %s failed", path);
}

int dotpe_bank_open(dotpe_ctx *ctx, const char *path, uint64_t *bank_id) {
  if (!ctx || !path || !bank_id) return fail(DOTPE_E_INVALID, "null argument");
  FILE *fp = fopen(path, "rb");
  if (!fp) return fail(DOTPE_E_INVALID, "cannot open %s", path);
  BankFileHeader h;
  if (fread(&h, sizeof(h), 1, fp) != 1 || memcmp(h.magic, BANK_MAGIC, 8) != 0 || h.version != BANK_VERSION) {
    fclose(fp);
    return fail(DOTPE_E_INVALID, "%s is not a bank file of this version", path);
  }
  // the ranges dotpe_bank_load accepts: n_pol 1 or 2, increasing mode numbers in 1..4
  bool modes_ok = h.n_modes >= 1 && h.n_modes <= MAXM;
  for (int m = 0; modes_ok && m < MAXM; ++m) {
    if (m < h.n_modes)
      modes_ok = h.mode_m[m] >= 1 && h.mode_m[m] <= 4 && (m == 0 || h.mode_m[m] > h.mode_m[m - 1]);
    else
      modes_ok = h.mode_m[m] == 0;
  }
  const int np = (int)h.n_pol;
  const bool shape_ok = modes_ok && (h.n_pol == 1 || h.n_pol == 2) && (h.has_lw == 0 || h.has_lw == 1) &&
                        (h.has_pol == 0 || h.has_pol == 1) && h.n_int >= 1 && h.n_bins >= 2 &&
                        h.kpad == (int)(((2 * np * (int64_t)h.n_bins + 63) / 64) * 64) && h.a_scale > 0.f &&
                        std::isfinite(h.a_scale);
  const size_t want = (size_t)h.n_bins * 16 + (h.has_lw ? (size_t)h.n_int * 8 : 0) +
                      (size_t)h.n_modes * h.n_int * h.kpad * 4 + (h.has_pol ? (size_t)h.n_int * h.n_modes * 16 : 0);
  if (!shape_ok || h.payload_bytes != want) {
    fclose(fp);
    return fail(DOTPE_E_INVALID, "%s: inconsistent header", path);
  }
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (cudaSetDevice(ctx->device) != cudaSuccess) {
    fclose(fp);
    return fail(DOTPE_E_DEVICE, "cudaSetDevice");
  }
  Bank *b = nullptr;
  uint8_t *extra = nullptr;  // 16 bytes of device scratch: amax and the plane scale
  int rc = bank_alloc(ctx, h.n_int, h.n_modes, h.n_bins, h.kpad, np, h.has_lw, h.has_pol, 16, &b, &extra);
  if (rc != DOTPE_OK) {
    fclose(fp);
    return rc;
  }
  for (int m = 0; m < MAXM; ++m) b->mode_m[m] = h.mode_m[m];
  b->a_scale = h.a_scale;
  struct Part { void *dst; size_t n; };
  const Part parts[5] = {{b->f, (size_t)b->B * 8}, {b->w, (size_t)b->B * 8}, {b->lw, b->lw ? (size_t)b->I * 8 : 0},
                         {b->master, (size_t)b->M * b->I * b->Kpad * 4},
                         {b->pol, b->pol ? (size_t)b->I * b->M * 16 : 0}};
  const size_t chunk = (size_t)64 << 20;
  std::vector<uint8_t> buf(chunk);
  uint64_t sum = header_hash(h);
  bool ok = true;
  for (const Part &p : parts)
    for (size_t o = 0; ok && o < p.n; o += chunk) {
      const size_t n = std::min(chunk, p.n - o);
      ok = fread(buf.data(), 1, n, fp) == n;
      if (ok) {
        sum = fnv1a(sum, buf.data(), n);
        ok = cudaMemcpy((uint8_t *)p.dst + o, buf.data(), n, cudaMemcpyHostToDevice) == cudaSuccess;
      }
    }
  fclose(fp);
  if (!ok || sum != h.checksum) {
    cudaFree(b->block);
    delete b;
    return fail(DOTPE_E_INVALID, "%s: %s", path, ok ? "checksum mismatch" : "truncated or unreadable payload");
  }
  // the operand planes at the saved scale: an amax whose power-of-two scale is a_scale
  float *amax = (float *)extra;
  const float am = 0.75f / b->a_scale;
  cudaStream_t st = ctx->main_stream;
  int64_t nel = (int64_t)b->M * b->I * b->Kpad;
  bool dev_ok = cudaMemcpyAsync(amax, &am, 4, cudaMemcpyHostToDevice, st) == cudaSuccess;
  launch_master_to_planes(nel, b->master, amax, b->bf, b->hf, amax + 1, st);
  dev_ok = dev_ok && cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(st) == cudaSuccess;
  if (!dev_ok) {
    cudaFree(b->block);
    delete b;
    return fail(DOTPE_E_DEVICE, "bank open: operand planes");
  }
  b->id = ctx->next_id++;
  ctx->banks[b->id] = b;
  ctx->used += b->bytes;
  *bank_id = b->id;
  return DOTPE_OK;
}

int dotpe_bank_subset(dotpe_ctx *ctx, uint64_t bank_id, const int64_t *rows, int64_t n, uint64_t *new_bank_id) {
  if (!ctx || !rows || !new_bank_id) return fail(DOTPE_E_INVALID, "null argument");
  if (n < 1) return fail(DOTPE_E_INVALID, "n=%lld rows", (long long)n);
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->banks.find(bank_id);
  if (it == ctx->banks.end()) return fail(DOTPE_E_NOT_FOUND, "bank %llu", (unsigned long long)bank_id);
  const Bank &s = *it->second;
  CUDA_OR_FAIL(cudaSetDevice(ctx->device));
  // the row list on the host, checked
  std::vector<int64_t> hr((size_t)n);
  if (is_device_ptr(rows)) CUDA_OR_FAIL(cudaMemcpy(hr.data(), rows, (size_t)n * 8, cudaMemcpyDeviceToHost));
  else memcpy(hr.data(), rows, (size_t)n * 8);
  for (int64_t r = 0; r < n; ++r)
    if (hr[r] < 0 || hr[r] >= s.I) return fail(DOTPE_E_INVALID, "rows[%lld]=%lld not in [0, %lld)", (long long)r,
                                                (long long)hr[r], (long long)s.I);
  Bank *b = new Bank();
  b->I = n;
  b->M = s.M;
  b->B = s.B;
  b->Kpad = s.Kpad;
  b->n_pol = s.n_pol;
  b->a_scale = s.a_scale;
  for (int m = 0; m < MAXM; ++m) b->mode_m[m] = s.mode_m[m];
  const size_t nel = (size_t)b->M * n * b->Kpad;
  Carver c;
  size_t o_f = c.take<double>(b->B), o_w = c.take<double>(b->B), o_lw = c.take<double>(s.lw ? n : 0);
  size_t o_master = c.take<float>(nel), o_bf = c.take<__nv_bfloat16>(2 * nel), o_hf = c.take<__half>(2 * nel);
  size_t o_pol = c.take<float2>(s.pol ? (size_t)n * b->M * 2 : 0);
  size_t o_rows = c.take<int64_t>(n);
  b->bytes = c.off;
  if (ctx->used + b->bytes > ctx->budget) {
    delete b;
    return fail(DOTPE_E_NOMEM, "bank subset needs %zu bytes beyond the budget", c.off);
  }
  if (cudaMalloc(&b->block, b->bytes) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return fail(DOTPE_E_NOMEM, "bank subset allocation of %zu bytes", c.off);
  }
  uint8_t *base = (uint8_t *)b->block;
  b->f = (double *)(base + o_f);
  b->w = (double *)(base + o_w);
  b->lw = s.lw ? (double *)(base + o_lw) : nullptr;
  b->master = (float *)(base + o_master);
  b->bf = (__nv_bfloat16 *)(base + o_bf);
  b->hf = (__half *)(base + o_hf);
  b->pol = s.pol ? (float2 *)(base + o_pol) : nullptr;
  int64_t *drows = (int64_t *)(base + o_rows);
  cudaStream_t st = ctx->main_stream;
  int rc = DOTPE_OK;
  auto check = [&](cudaError_t x) {
    if (x != cudaSuccess && rc == DOTPE_OK) rc = fail(DOTPE_E_DEVICE, "bank subset: %s", cudaGetErrorString(x));
  };
  check(cudaMemcpyAsync(drows, hr.data(), (size_t)n * 8, cudaMemcpyHostToDevice, st));
  check(cudaMemcpyAsync(b->f, s.f, (size_t)b->B * 8, cudaMemcpyDeviceToDevice, st));
  check(cudaMemcpyAsync(b->w, s.w, (size_t)b->B * 8, cudaMemcpyDeviceToDevice, st));
  // the same operand values row by row (planes keep the parent's scale)
  const int64_t kw = b->Kpad;  // words per master row; a plane row is Kpad 16-bit values = Kpad / 2 words
  launch_gather_rows(b->M, s.I, n, kw, s.master, drows, b->master, st);
  launch_gather_rows(2 * b->M, s.I, n, kw / 2, s.bf, drows, b->bf, st);
  launch_gather_rows(2 * b->M, s.I, n, kw / 2, s.hf, drows, b->hf, st);
  if (s.lw) launch_gather_rows(1, s.I, n, 2, s.lw, drows, b->lw, st);
  if (s.pol) launch_gather_rows(1, s.I, n, 4 * b->M, s.pol, drows, b->pol, st);
  check(cudaGetLastError());
  check(cudaStreamSynchronize(st));
  if (rc != DOTPE_OK) {
    cudaFree(b->block);
    delete b;
    return rc;
  }
  b->id = ctx->next_id++;
  ctx->banks[b->id] = b;
  ctx->used += b->bytes;
  *new_bank_id = b->id;
  return DOTPE_OK;
}

int dotpe_bank_release(dotpe_ctx *ctx, uint64_t bank_id) {
  if (!ctx) return fail(DOTPE_E_INVALID, "ctx is null");
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->banks.find(bank_id);
  if (it == ctx->banks.end()) return fail(DOTPE_E_NOT_FOUND, "bank %llu", (unsigned long long)bank_id);
  if (it->second->refs > 0) return fail(DOTPE_E_INVALID, "bank still used by %d events", it->second->refs);
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  for (XEntry *x : it->second->xcache) {
    cudaFree(x->mx);
    cudaEventDestroy(x->ready);
    ctx->used -= x->bytes;
    delete x;
  }
  cudaFree(it->second->block);
  ctx->used -= it->second->bytes;
  delete it->second;
  ctx->banks.erase(it);
  return DOTPE_OK;
}

}  // extern "C"

// Validates one descriptor, copies its inputs into device memory and queues the
// event (caller holds ctx->mu).  group != 0 marks the events of one batch.
static int submit_locked(dotpe_ctx *ctx, const dotpe_event_desc *d, uint64_t group, uint64_t *event_id) {
  if (!d) return fail(DOTPE_E_INVALID, "null descriptor");
  auto bit = ctx->banks.find(d->bank_id);
  if (bit == ctx->banks.end()) return fail(DOTPE_E_NOT_FOUND, "bank %llu", (unsigned long long)d->bank_id);
  Bank *b = bit->second;
  if (d->i0 < 0 || d->i1 <= d->i0 || d->i1 > b->I) return fail(DOTPE_E_INVALID, "slice [%lld,%lld) of %lld rows",
                                                               (long long)d->i0, (long long)d->i1, (long long)b->I);
  if (d->n_det < 1 || d->n_det > MAXD) return fail(DOTPE_E_INVALID, "n_det=%d not in 1..%d", d->n_det, MAXD);
  if (d->n_ext < 1) return fail(DOTPE_E_INVALID, "n_ext=%lld", (long long)d->n_ext);
  if (d->n_phi < 1 || d->n_phi > MAXPHI) return fail(DOTPE_E_INVALID, "n_phi=%d not in 1..%d", d->n_phi, MAXPHI);
  if (!(d->u_min > 0.0) || !std::isfinite(d->u_min)) return fail(DOTPE_E_INVALID, "u_min must be > 0");
  const bool rb = d->rb_dh || d->rb_hh;
  const bool pol = (b->n_pol == 2);
  if (rb && !(d->rb_dh && d->rb_hh)) return fail(DOTPE_E_INVALID, "rb_dh and rb_hh go together");
  if ((!rb && (!d->psd || !d->data)) || !d->t || (pol ? !d->F : !d->R))
    return fail(DOTPE_E_INVALID, pol ? "null input array (a polarisation-resolved bank needs F)" : "null input array");
  if (pol && d->precision != DOTPE_PREC_FP32 && d->n_det > POL_TC_MAXD)
    return fail(DOTPE_E_UNSUPPORTED, "a polarisation-resolved bank with n_det=%d runs in FP32 only (tensor cores: "
                "n_det <= %d)", d->n_det, POL_TC_MAXD);
  if (!rb && (size_t)d->n_det * b->B * sizeof(float) > 227 * 1024)
    return fail(DOTPE_E_UNSUPPORTED, "n_det * n_bins = %lld: the <h|h> weights exceed shared memory",
                (long long)d->n_det * b->B);
  if (d->precision < DOTPE_PREC_FP32 || d->precision > DOTPE_PREC_MIXED)
    return fail(DOTPE_E_INVALID, "precision %d", d->precision);
  if (d->block_rows < 0 || d->block_rows % TC_TI != 0)
    return fail(DOTPE_E_INVALID, "block_rows=%lld is not a non-negative multiple of %d", (long long)d->block_rows, TC_TI);
  const int64_t NI = d->i1 - d->i0, NE = d->n_ext;
  if (d->precision != DOTPE_PREC_FP32 && (2 * (int64_t)b->M * 2 * NE >= (1ll << 31)))
    return fail(DOTPE_E_UNSUPPORTED, "n_ext too large");
  Event *e = new Event();
  e->bank = b;
  e->i0 = d->i0;
  e->NI = NI;
  e->NE = NE;
  e->D = d->n_det;
  e->nphi = d->n_phi;
  e->prec = d->precision;
  e->block_rows = d->block_rows;
  e->flags = d->flags;
  e->u_min = d->u_min;
  e->cut = d->cut_delta;
  e->has_lwe = d->ln_w_ext != nullptr;
  e->group = group;
  // footprint check against the whole budget
  size_t need = scratch_layout(*e).total + keep_bytes_of(*e);
  Carver c;
  const int64_t D = e->D, B = b->B, M = b->M;
  const int64_t J = M * b->n_pol;  // relative-binning components (mode, polarisation)
  size_t o_psd = c.take<double>(D * B), o_data = c.take<double2>(D * B), o_t = c.take<double>(NE * D);
  size_t o_R = c.take<double2>(NE * D * M), o_lw = c.take<double>(NE);
  size_t o_rbd = c.take<double2>(rb ? D * J * B : 0), o_rbh = c.take<double2>(rb ? D * J * J * B : 0);
  size_t o_F = c.take<double>(pol ? NE * D * 2 : 0);
  e->in_bytes = c.off;
  if (need + e->in_bytes + b->bytes > ctx->budget) {
    delete e;
    return fail(DOTPE_E_ADMISSION, "event needs %zu device bytes, budget %llu", need + c.off,
                (unsigned long long)ctx->budget);
  }
  // device copy of the inputs, ordered after the caller's stream
  cudaStream_t ist = ctx->input_stream;
  auto cleanup = [&](int rc) {
    if (e->in_block) cudaFree(e->in_block);
    if (e->in_stage) cudaFreeHost(e->in_stage);
    delete e;
    return rc;
  };
  if (cudaMallocAsync(&e->in_block, e->in_bytes, ist) != cudaSuccess) {
    cudaGetLastError();
    delete e;
    return fail(DOTPE_E_NOMEM, "event inputs");
  }
  uint8_t *ib = (uint8_t *)e->in_block;
  e->psd = (double *)(ib + o_psd);
  e->data = (double2 *)(ib + o_data);
  e->t = (double *)(ib + o_t);
  e->R = (double2 *)(ib + o_R);
  e->lwe = (double *)(ib + o_lw);
  if (rb) {
    e->rb_dh = (double2 *)(ib + o_rbd);
    e->rb_hh = (double2 *)(ib + o_rbh);
  }
  if (pol) e->F = (double *)(ib + o_F);
  struct Piece { const void *src; void *dst; size_t n; };
  Piece pieces[8] = {{d->psd, e->psd, d->psd ? (size_t)(D * B * 8) : 0},
                     {d->data, e->data, d->data ? (size_t)(D * B * 16) : 0},
                     {d->t, e->t, (size_t)(NE * D * 8)},
                     {d->R, e->R, (!pol && d->R) ? (size_t)(NE * D * M * 16) : 0},
                     {d->F, e->F, pol ? (size_t)(NE * D * 2 * 8) : 0},
                     {d->ln_w_ext, e->lwe, d->ln_w_ext ? (size_t)(NE * 8) : 0},
                     {d->rb_dh, e->rb_dh, rb ? (size_t)(D * J * B * 16) : 0},
                     {d->rb_hh, e->rb_hh, rb ? (size_t)(D * J * J * B * 16) : 0}};
  size_t host_total = 0;
  for (auto &p : pieces)
    if (p.n && !is_device_ptr(p.src)) host_total += p.n;
  if (host_total) {
    if (cudaHostAlloc(&e->in_stage, host_total, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return cleanup(fail(DOTPE_E_NOMEM, "pinned staging"));
    }
    e->stage_bytes = host_total;
  }
  if (d->stream) {
    cudaEvent_t dep;
    cudaEventCreateWithFlags(&dep, cudaEventDisableTiming);
    cudaEventRecord(dep, (cudaStream_t)d->stream);
    cudaStreamWaitEvent(ist, dep, 0);
    cudaEventDestroy(dep);
  }
  size_t so = 0;
  for (auto &p : pieces) {
    if (!p.n) continue;
    if (is_device_ptr(p.src)) {
      if (copy_in(p.dst, p.src, p.n, ist) != DOTPE_OK) return cleanup(DOTPE_E_DEVICE);
    } else {
      uint8_t *hs = (uint8_t *)e->in_stage + so;
      memcpy(hs, p.src, p.n);
      so += p.n;
      if (copy_in(p.dst, hs, p.n, ist) != DOTPE_OK) return cleanup(DOTPE_E_DEVICE);
    }
  }
  {
    int rc = rb ? psd_hash(e->D, (int)B, nullptr, &e->psd_key, d->rb_hh, (size_t)(2 * D * J * J * B))
                : psd_hash(e->D, (int)B, d->psd, &e->psd_key);
    if (rc != DOTPE_OK) return cleanup(rc);
  }
  cudaEventCreateWithFlags(&e->ev_inputs, cudaEventDisableTiming);
  cudaEventCreate(&e->ev_start);
  cudaEventCreate(&e->ev_end);
  cudaEventCreate(&e->ev_k0);
  cudaEventCreate(&e->ev_k1);
  cudaEventCreate(&e->ev_ks);
  cudaEventRecord(e->ev_inputs, ist);
  if (cudaHostAlloc((void **)&e->h_out, sizeof(ReduceOut), cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    return cleanup(fail(DOTPE_E_NOMEM, "pinned result"));
  }
  memset(e->h_out, 0, sizeof(ReduceOut));
  e->id = ctx->next_id++;
  e->t_submit = now_ns();
  b->refs++;
  ctx->used += e->in_bytes;
  ctx->events[e->id] = e;
  ctx->queue.push_back(e->id);
  *event_id = e->id;
  return DOTPE_OK;
}

extern "C" {

int dotpe_event_submit(dotpe_ctx *ctx, const dotpe_event_desc *d, uint64_t *event_id) {
  if (!ctx || !d || !event_id) return fail(DOTPE_E_INVALID, "null argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  CUDA_OR_FAIL(cudaSetDevice(ctx->device));
  int rc = submit_locked(ctx, d, 0, event_id);
  if (rc != DOTPE_OK) return rc;
  progress(ctx);
  Event *e = ctx->events[*event_id];
  if (e->state == DOTPE_STATE_FAILED) return fail(DOTPE_E_DEVICE, "launch failed: %s", g_last_error.c_str());
  return DOTPE_OK;
}

int dotpe_batch_submit(dotpe_ctx *ctx, int n, const dotpe_event_desc *descs, uint64_t *event_ids) {
  if (!ctx || !descs || !event_ids || n < 1) return fail(DOTPE_E_INVALID, "null argument or n < 1");
  std::lock_guard<std::mutex> lk(ctx->mu);
  CUDA_OR_FAIL(cudaSetDevice(ctx->device));
  for (int k = 1; k < n; ++k)
    if (descs[k].bank_id != descs[0].bank_id || descs[k].precision != descs[0].precision)
      return fail(DOTPE_E_INVALID, "batch events must share the bank and the precision");
  {
    auto bit = ctx->banks.find(descs[0].bank_id);
    if (bit != ctx->banks.end() && bit->second->n_pol == 2 && descs[0].precision != DOTPE_PREC_FP32)
      return fail(DOTPE_E_UNSUPPORTED, "batches of a polarisation-resolved bank run in FP32 only");
  }
  size_t need = 0;
  const uint64_t group = ctx->next_group++;
  for (int k = 0; k < n; ++k) {
    if (descs[k].block_rows != 0) return fail(DOTPE_E_INVALID, "batch events are not streamed in bank blocks");
    int rc = submit_locked(ctx, &descs[k], group, &event_ids[k]);
    if (rc != DOTPE_OK) {
      std::string msg = g_last_error;
      for (int j = 0; j < k; ++j) {
        auto it = ctx->events.find(event_ids[j]);
        ctx->queue.erase(std::remove(ctx->queue.begin(), ctx->queue.end(), event_ids[j]), ctx->queue.end());
        free_event(ctx, it->second);
        ctx->events.erase(it);
      }
      return fail(rc, "batch event %d: %s", k, msg.c_str());
    }
    Event *e = ctx->events[event_ids[k]];
    need += scratch_layout(*e).total + keep_bytes_of(*e) + e->in_bytes;
  }
  if (need + ctx->events[event_ids[0]]->bank->bytes > ctx->budget) {
    for (int j = 0; j < n; ++j) {
      auto it = ctx->events.find(event_ids[j]);
      ctx->queue.erase(std::remove(ctx->queue.begin(), ctx->queue.end(), event_ids[j]), ctx->queue.end());
      free_event(ctx, it->second);
      ctx->events.erase(it);
    }
    return fail(DOTPE_E_ADMISSION, "batch needs %zu device bytes, budget %llu", need,
                (unsigned long long)ctx->budget);
  }
  progress(ctx);
  for (int k = 0; k < n; ++k)
    if (ctx->events[event_ids[k]]->state == DOTPE_STATE_FAILED)
      return fail(DOTPE_E_DEVICE, "launch failed: %s", g_last_error.c_str());
  return DOTPE_OK;
}

static void fill_stats(const Event &e, dotpe_event_stats *s) {
  if (!s) return;
  s->t_submit_ns = e.t_submit;
  s->t_admit_ns = e.t_admit;
  s->t_done_ns = e.t_done;
  s->n_pairs = e.NI * e.NE;
  s->footprint_bytes = (int64_t)(e.keep_bytes + scratch_layout(e, e.want_hb).total + e.in_bytes);
  s->device_ms = e.device_ms;
  s->prep_ms = e.prep_ms;
  s->fused_ms = e.fused_ms;
  s->refine_ms = e.refine_ms;
  s->precision = e.prec;
  s->state = e.state;
}

int dotpe_event_poll(dotpe_ctx *ctx, uint64_t event_id, int *state, dotpe_event_stats *stats) {
  if (!ctx) return fail(DOTPE_E_INVALID, "ctx is null");
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  progress(ctx);
  auto it = ctx->events.find(event_id);
  if (it == ctx->events.end()) return fail(DOTPE_E_NOT_FOUND, "event %llu", (unsigned long long)event_id);
  if (state) *state = it->second->state;
  fill_stats(*it->second, stats);
  return DOTPE_OK;
}

int dotpe_event_wait(dotpe_ctx *ctx, uint64_t event_id, double timeout_s) {
  if (!ctx) return fail(DOTPE_E_INVALID, "ctx is null");
  const int64_t t0 = now_ns();
  while (true) {
    {
      std::lock_guard<std::mutex> lk(ctx->mu);
      cudaSetDevice(ctx->device);
      progress(ctx);
      auto it = ctx->events.find(event_id);
      if (it == ctx->events.end()) return fail(DOTPE_E_NOT_FOUND, "event %llu", (unsigned long long)event_id);
      int s = it->second->state;
      if (s == DOTPE_STATE_DONE) return DOTPE_OK;
      if (s == DOTPE_STATE_FAILED) {
        int ds = it->second->h_out->status;
        int code = ds == DEV_E_NONFINITE ? DOTPE_E_INVALID : ds == DEV_E_TIMEOUT ? DOTPE_E_TIMEOUT : DOTPE_E_DEVICE;
        return fail(code, "event failed (device status %d%s%s)", ds, it->second->launch_error.empty() ? "" : "; ",
                    it->second->launch_error.c_str());
      }
    }
    if (timeout_s > 0 && (now_ns() - t0) > (int64_t)(timeout_s * 1e9)) return fail(DOTPE_E_TIMEOUT, "event wait");
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

int dotpe_event_stream_wait(dotpe_ctx *ctx, uint64_t event_id, void *stream) {
  if (!ctx) return fail(DOTPE_E_INVALID, "ctx is null");
  while (true) {
    {
      std::lock_guard<std::mutex> lk(ctx->mu);
      CUDA_OR_FAIL(cudaSetDevice(ctx->device));
      progress(ctx);
      auto it = ctx->events.find(event_id);
      if (it == ctx->events.end()) return fail(DOTPE_E_NOT_FOUND, "event %llu", (unsigned long long)event_id);
      Event &e = *it->second;
      if (e.state != DOTPE_STATE_QUEUED) {
        CUDA_OR_FAIL(cudaStreamWaitEvent((cudaStream_t)stream, e.ev_end, 0));
        return DOTPE_OK;
      }
    }
    // still queued: wait for an earlier event to finish and free its slot
    std::unique_lock<std::mutex> lk(ctx->cb_mu);
    ctx->cv.wait_for(lk, std::chrono::milliseconds(1));
  }
}

int dotpe_evidence(dotpe_ctx *ctx, uint64_t event_id, dotpe_evidence_out *out) {
  if (!ctx || !out) return fail(DOTPE_E_INVALID, "null argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  progress(ctx);
  auto it = ctx->events.find(event_id);
  if (it == ctx->events.end()) return fail(DOTPE_E_NOT_FOUND, "event %llu", (unsigned long long)event_id);
  Event &e = *it->second;
  if (e.state == DOTPE_STATE_QUEUED || e.state == DOTPE_STATE_RUNNING) return fail(DOTPE_E_NOT_READY, "event not done");
  const ReduceOut &r = *e.h_out;
  memset(out, 0, sizeof(*out));
  out->ln_z = r.ln_z;
  out->n_eff = r.n_eff;
  out->n_eff_int = r.n_eff_int;
  out->n_eff_ext = r.n_eff_ext;
  out->max_lnl_ml = r.max_ml;
  long long a = r.arg;
  out->arg_o = a % e.nphi;
  a /= e.nphi;
  out->arg_e = a % e.NE;
  out->arg_i = a / e.NE + e.i0;
  out->n_marginalised = r.n_marg;
  out->n_pairs = e.NI * e.NE;
  out->lnl_ml_threshold = r.threshold;
  out->device_status = r.status;
  out->n_refined_tiles = r.n_refined;
  out->n_screen_candidates = r.n_cand;
  out->n_screen_evaluated = r.n_eval;
  if (r.status == DEV_E_NONFINITE) return fail(DOTPE_E_INVALID, "non-finite or non-positive event input");
  if (r.status == DEV_E_TIMEOUT) return fail(DOTPE_E_TIMEOUT, "device wait timed out");
  if (r.status != 0) return fail(DOTPE_E_DEVICE, "device status %d", r.status);
  return DOTPE_OK;
}

}  // extern "C"

// Recomputes ln Lbar_ie or max_o ln L^ML_ie of rows [a, b) x samples [e0, e1)
// of a finished event that did not store them: a sub-event over that block with
// the event's inputs, in the event's arithmetic (split fp16 for the mixed
// path), with the ML cut fixed at the event's final threshold, run to
// completion on the context's main stream (caller holds ctx->mu).
static int recompute_block(dotpe_ctx *ctx, Event &e, int64_t a, int64_t b, int64_t e0, int64_t e1, int what,
                           float *out, int64_t ld) {
  Event sub;
  sub.id = 0;
  sub.bank = e.bank;
  sub.i0 = e.i0 + a;
  sub.NI = b - a;
  sub.NE = e1 - e0;
  sub.D = e.D;
  sub.nphi = e.nphi;
  sub.prec = (e.prec == DOTPE_PREC_MIXED) ? DOTPE_PREC_FP16X3 : e.prec;
  sub.flags = DOTPE_FLAG_STORE_LNL;
  sub.u_min = e.u_min;
  sub.cut = e.cut;
  sub.has_lwe = e.has_lwe;
  sub.psd = e.psd;
  sub.data = e.data;
  sub.rb_dh = e.rb_dh;
  sub.rb_hh = e.rb_hh;
  sub.F = e.F;
  sub.t = e.t + e0 * e.D;
  sub.R = e.R + e0 * e.D * e.bank->M;
  sub.lwe = e.lwe + e0;
  sub.in_block = e.in_block;
  sub.owns_inputs = false;
  sub.psd_key = e.psd_key;
  if (e.cut > 0) sub.frozen_max = (float)(e.h_out->threshold + e.cut);
  sub.slot = 0;
  CUDA_OR_FAIL(cudaEventCreateWithFlags(&sub.ev_inputs, cudaEventDisableTiming));
  CUDA_OR_FAIL(cudaEventCreate(&sub.ev_start));
  CUDA_OR_FAIL(cudaEventCreate(&sub.ev_end));
  CUDA_OR_FAIL(cudaEventCreate(&sub.ev_k0));
  CUDA_OR_FAIL(cudaEventCreate(&sub.ev_k1));
  CUDA_OR_FAIL(cudaEventCreate(&sub.ev_ks));
  CUDA_OR_FAIL(cudaHostAlloc((void **)&sub.h_out, sizeof(ReduceOut), cudaHostAllocDefault));
  cudaStream_t st = ctx->main_stream;
  CUDA_OR_FAIL(cudaEventRecord(sub.ev_inputs, st));
  int rc = DOTPE_OK;
  {
    EventRun R;
    rc = event_alloc(ctx, sub, st, R);
    if (rc == DOTPE_OK) {
      // cross terms of these rows: the cached entry of the bank for this PSD if there is one
      for (XEntry *c : sub.bank->xcache)
        if (c->key == sub.psd_key && c->D == sub.D) {
          CUDA_OR_FAIL(cudaStreamWaitEvent(st, c->ready, 0));
          sub.xent = c;
        }
      if ((rc = event_begin(sub, R, st)) == DOTPE_OK) {
        event_block(ctx, sub, R, 0, sub.NI, st);
        rc = event_fused(ctx, sub, R, true, st);
      }
      cudaFreeAsync(R.scr, st);
    }
  }
  if (rc == DOTPE_OK) {
    CUDA_OR_FAIL(cudaStreamSynchronize(st));
    const float *src = (what == DOTPE_LNL_MARG) ? sub.lnl_tile : sub.ml_tile;
    cudaError_t ce = cudaMemcpy2D(out, ld * 4, src, sub.NE * 4, sub.NE * 4, sub.NI, cudaMemcpyDefault);
    if (ce != cudaSuccess) rc = fail(DOTPE_E_DEVICE, "copying the recomputed block: %s", cudaGetErrorString(ce));
  } else {
    cudaStreamSynchronize(st);
  }
  if (sub.keep_block) cudaFree(sub.keep_block);
  cudaFreeHost(sub.h_out);
  cudaEventDestroy(sub.ev_inputs);
  cudaEventDestroy(sub.ev_start);
  cudaEventDestroy(sub.ev_end);
  cudaEventDestroy(sub.ev_k0);
  cudaEventDestroy(sub.ev_k1);
  cudaEventDestroy(sub.ev_ks);
  return rc;
}

extern "C" {

int dotpe_lnl_blocks(dotpe_ctx *ctx, uint64_t event_id, int64_t i0, int64_t i1, int64_t e0, int64_t e1, int what,
                     float *out, int64_t ld) {
  if (!ctx || !out) return fail(DOTPE_E_INVALID, "null argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  CUDA_OR_FAIL(cudaSetDevice(ctx->device));
  progress(ctx);
  auto it = ctx->events.find(event_id);
  if (it == ctx->events.end()) return fail(DOTPE_E_NOT_FOUND, "event %llu", (unsigned long long)event_id);
  Event &e = *it->second;
  if (e.state != DOTPE_STATE_DONE) return fail(DOTPE_E_NOT_READY, "event not done");
  if (what == DOTPE_LNL_MARG || what == DOTPE_LNL_ML_MAX) {
    if (i0 < 0 || i1 > e.NI || i1 <= i0 || e0 < 0 || e1 > e.NE || e1 <= e0 || ld < e1 - e0)
      return fail(DOTPE_E_INVALID, "block range");
    if (!(e.flags & DOTPE_FLAG_STORE_LNL)) return recompute_block(ctx, e, i0, i1, e0, e1, what, out, ld);
    const float *src = (what == DOTPE_LNL_MARG ? e.lnl_tile : e.ml_tile) + i0 * e.NE + e0;
    CUDA_OR_FAIL(cudaMemcpy2D(out, ld * 4, src, e.NE * 4, (e1 - e0) * 4, i1 - i0, cudaMemcpyDefault));
    return DOTPE_OK;
  }
  if (what == DOTPE_ROW_MARGINAL || what == DOTPE_COL_MARGINAL) {
    const bool row = what == DOTPE_ROW_MARGINAL;
    int64_t a = row ? i0 : e0, z = row ? i1 : e1, n = row ? e.NI : e.NE;
    if (a < 0 || z > n || z <= a) return fail(DOTPE_E_INVALID, "marginal range");
    std::vector<double> tmp(z - a);
    CUDA_OR_FAIL(cudaMemcpy(tmp.data(), (row ? e.ln_p_int : e.ln_p_ext) + a, (z - a) * 8, cudaMemcpyDeviceToHost));
    std::vector<float> f(z - a);
    for (size_t k = 0; k < f.size(); ++k) f[k] = (float)tmp[k];
    CUDA_OR_FAIL(cudaMemcpy(out, f.data(), f.size() * 4, cudaMemcpyDefault));
    return DOTPE_OK;
  }
  return fail(DOTPE_E_INVALID, "what=%d", what);
}

int dotpe_posterior_samples(dotpe_ctx *ctx, uint64_t event_id, int64_t n, const double *uniforms, int64_t *i_out,
                            int64_t *e_out, int32_t *o_out, double *dist_out) {
  if (!ctx) return fail(DOTPE_E_INVALID, "ctx is null");
  std::lock_guard<std::mutex> lk(ctx->mu);
  CUDA_OR_FAIL(cudaSetDevice(ctx->device));
  progress(ctx);
  auto it = ctx->events.find(event_id);
  if (it == ctx->events.end()) return fail(DOTPE_E_NOT_FOUND, "event %llu", (unsigned long long)event_id);
  Event &e = *it->second;
  if (e.state != DOTPE_STATE_DONE) return fail(DOTPE_E_NOT_READY, "event not done");
  return samples_locked(ctx, e, n, uniforms, i_out, e_out, o_out, dist_out);
}

int dotpe_rb_weights(dotpe_ctx *ctx, const dotpe_rb_desc *desc, double *w_dh, double *w_hh) {
  if (!ctx || !desc) return fail(DOTPE_E_INVALID, "null argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  CUDA_OR_FAIL(cudaSetDevice(ctx->device));
  return rb_weights_locked(ctx, desc, w_dh, w_hh);
}

int dotpe_preselect(dotpe_ctx *ctx, const dotpe_presel_desc *desc, float *lnl_ml, int32_t *arg_ot,
                    double *lnl_inco, int64_t *selected, dotpe_presel_out *out) {
  if (!ctx || !desc) return fail(DOTPE_E_INVALID, "null argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  CUDA_OR_FAIL(cudaSetDevice(ctx->device));
  return preselect_locked(ctx, desc, lnl_ml, arg_ot, lnl_inco, selected, out);
}

int dotpe_event_release(dotpe_ctx *ctx, uint64_t event_id) {
  if (!ctx) return fail(DOTPE_E_INVALID, "ctx is null");
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  auto it = ctx->events.find(event_id);
  if (it == ctx->events.end()) return fail(DOTPE_E_NOT_FOUND, "event %llu", (unsigned long long)event_id);
  Event *e = it->second;
  if (e->state == DOTPE_STATE_RUNNING) {
    cudaEventSynchronize(e->ev_end);
    progress(ctx);
  }
  for (auto q = ctx->queue.begin(); q != ctx->queue.end(); ++q)
    if (*q == event_id) {
      ctx->queue.erase(q);
      break;
    }
  ctx->events.erase(it);
  free_event(ctx, e);
  progress(ctx);
  return DOTPE_OK;
}

int dotpe_dist_marg_eval(dotpe_ctx *ctx, int64_t n, const float *dh, const float *hh, float u_min, float *out) {
  if (!ctx || !dh || !hh || !out || n < 0) return fail(DOTPE_E_INVALID, "null argument");
  if (n == 0) return DOTPE_OK;
  std::lock_guard<std::mutex> lk(ctx->mu);
  CUDA_OR_FAIL(cudaSetDevice(ctx->device));
  float *buf = nullptr;
  CUDA_OR_FAIL(cudaMalloc(&buf, 3 * n * sizeof(float)));
  cudaStream_t st = ctx->main_stream;
  cudaMemcpyAsync(buf, dh, n * 4, cudaMemcpyDefault, st);
  cudaMemcpyAsync(buf + n, hh, n * 4, cudaMemcpyDefault, st);
  launch_dist_marg_eval(n, buf, buf + n, u_min, ctx->dm_table, buf + 2 * n, st);
  cudaMemcpyAsync(out, buf + 2 * n, n * 4, cudaMemcpyDefault, st);
  cudaError_t e = cudaStreamSynchronize(st);
  cudaFree(buf);
  if (e != cudaSuccess) return fail(DOTPE_E_DEVICE, "%s", cudaGetErrorString(e));
  return DOTPE_OK;
}

int dotpe_evidence_merge(int n_shards, const dotpe_shard *shards, int64_t n_ext, int n_phi,
                         dotpe_evidence_out *out, double *ln_p_ext_out) {
  if (!shards || !out) return fail(DOTPE_E_INVALID, "null argument");
  if (n_shards < 1 || n_ext < 1 || n_phi < 1)
    return fail(DOTPE_E_INVALID, "n_shards=%d n_ext=%lld n_phi=%d", n_shards, (long long)n_ext, n_phi);
  for (int r = 0; r < n_shards; ++r)
    if (shards[r].n_int < 1 || !shards[r].ln_p_ext) return fail(DOTPE_E_INVALID, "shard %d: n_int or ln_p_ext", r);
  // log-sum-exp accumulator in FP64
  struct L {
    double m = -INFINITY, s = 0.0;
    void add(double x) {
      if (x == -INFINITY) return;
      if (x > m) { s = s * std::exp(m - x) + 1.0; m = x; }
      else s += std::exp(x - m);
    }
    double val() const { return s > 0.0 ? m + std::log(s) : -INFINITY; }
  };
  L s1, s2, spi;
  int64_t n_int = 0;
  dotpe_evidence_out o;
  memset(&o, 0, sizeof(o));
  o.max_lnl_ml = -INFINITY;
  o.lnl_ml_threshold = -INFINITY;
  bool refined = true, screened = true;
  for (int r = 0; r < n_shards; ++r) {
    const dotpe_evidence_out &e = shards[r].ev;
    const double ls1 = e.ln_z + std::log((double)shards[r].n_int) + std::log((double)n_ext) +
                       std::log((double)n_phi);
    if (ls1 != -INFINITY && e.n_eff > 0.0) {
      s1.add(ls1);
      s2.add(2.0 * ls1 - std::log(e.n_eff));             // sum p^2 of the shard
      if (e.n_eff_int > 0.0) spi.add(2.0 * ls1 - std::log(e.n_eff_int));  // sum_i P_i^2
    }
    n_int += shards[r].n_int;
    if (e.max_lnl_ml > o.max_lnl_ml ||
        (e.max_lnl_ml == o.max_lnl_ml &&
         (e.arg_i < o.arg_i || (e.arg_i == o.arg_i && (e.arg_e < o.arg_e || (e.arg_e == o.arg_e && e.arg_o < o.arg_o)))))) {
      o.max_lnl_ml = e.max_lnl_ml;
      o.arg_i = e.arg_i;
      o.arg_e = e.arg_e;
      o.arg_o = e.arg_o;
    }
    o.n_marginalised += e.n_marginalised;
    o.n_pairs += e.n_pairs;
    o.lnl_ml_threshold = std::max(o.lnl_ml_threshold, e.lnl_ml_threshold);
    if (o.device_status == 0) o.device_status = e.device_status;
    if (e.n_refined_tiles < 0) refined = false;
    else o.n_refined_tiles += e.n_refined_tiles;
    if (e.n_screen_candidates < 0 || e.n_screen_evaluated < 0) screened = false;
    o.n_screen_candidates += e.n_screen_candidates;
    o.n_screen_evaluated += e.n_screen_evaluated;
  }
  if (!refined) o.n_refined_tiles = -1;
  if (!screened) o.n_screen_candidates = o.n_screen_evaluated = -1;
  // per-sample marginals: the shards' sums added, then sum_e P_e^2
  L spe;
  for (int64_t k = 0; k < n_ext; ++k) {
    L pe;
    for (int r = 0; r < n_shards; ++r) pe.add(shards[r].ln_p_ext[k]);
    const double v = pe.val();
    if (ln_p_ext_out) ln_p_ext_out[k] = v;
    if (v != -INFINITY) spe.add(2.0 * v);
  }
  const double l1 = s1.val();
  o.ln_z = l1 - std::log((double)n_int) - std::log((double)n_ext) - std::log((double)n_phi);
  o.n_eff = (l1 == -INFINITY) ? 0.0 : std::exp(2.0 * l1 - s2.val());
  o.n_eff_int = (l1 == -INFINITY) ? 0.0 : std::exp(2.0 * l1 - spi.val());
  o.n_eff_ext = (l1 == -INFINITY) ? 0.0 : std::exp(2.0 * l1 - spe.val());
  *out = o;
  return DOTPE_OK;
}

int dotpe_dist_marg_eval_noalloc(dotpe_ctx *ctx, int64_t n, const float *dh, const float *hh, float u_min,
                                  float *out) {
  if (!ctx || (n > 0 && (!dh || !hh || !out))) return fail(DOTPE_E_INVALID, "null argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  CUDA_OR_FAIL(cudaSetDevice(ctx->device));
  char msg[256] = {0};
  int rc = dist_marg_eval_noalloc(ctx->device, n, dh, hh, u_min, ctx->dm_table, out, ctx->main_stream, msg,
                                  sizeof(msg));
  if (rc != DOTPE_OK) return fail(rc, "%s", msg);
  return DOTPE_OK;
}

}  // extern "C"
