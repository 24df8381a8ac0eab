// Internal definitions shared by the dotpe CUDA translation units (sm_103a).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dotpe.h"

namespace dotpe {

constexpr int MAXM = 4;    // modes per waveform
constexpr int MAXD = 3;    // detectors (H, L, V)
constexpr int REC = 16;    // floats per (row or column, detector) cross-term record
constexpr int REC_P = 24;  // row record of a polarisation-resolved bank (21 used, see cross_terms_pol_kernel)
constexpr int REC_POL = 21;     // used floats of that record
constexpr int POL_TC_MAXD = 3;  // detectors of a polarisation-resolved bank on the tensor cores (registers)
constexpr int MAXPHI = 128;
constexpr int NPAIR = 6;   // mode pairs (a > b) for MAXM = 4

// Device error codes written into an event's status word (never __trap()).
enum : int {
  DEV_OK = 0,
  DEV_E_NONFINITE = 1,     // NaN/Inf/non-positive PSD in the event inputs
  DEV_E_TIMEOUT = 2,       // a bounded mbarrier wait ran out
  DEV_E_SHAPE = 3,
};

// Everything the fused epilogue needs besides the per-pair GEMM outputs.
struct EpiParams {
  int n_modes, n_det, n_phi;
  int mode_m[MAXM];
  int npair;                // n_modes (n_modes - 1) / 2
  int pdelta[NPAIR];        // m_a - m_b of pair p (index into C_delta, 1..3)
  int consec;               // azimuthal numbers are consecutive: pdelta[p] = a - b
  float u_min;
  float z_scale;            // accumulator -> <d|h> component scale (times 1 / *g_scale)
  const float *g_scale;     // device scale applied to the extrinsic operand (null: 1)
  float cut_delta;          // > 0: coherent-ML selection on
  float ln_nphi;
  int64_t n_int, n_ext;     // slice sizes
  int64_t i_base;           // first bank row of the slice
  const float *mx;          // [n_int][n_det][REC] row cross-term records (slice-relative)
  const float *qx;          // [n_ext][n_det][REC] column records
  const double *lw_int;     // [n_int] slice-relative, may be null
  const double *lw_ext;     // [n_ext], may be null
  const float4 *dm_table;   // distance-marginal Hermite table
  float *ml_running;        // running max of ln L^ML (>= 0)
  int track_max;            // raise *ml_running with each tile's best ln L^ML
  int screen_ml;            // screening pass: max_o ln L^ML only (no distance marginal)
  float margin_k;           // screening error scale kappa*u (0: exact threshold)
  const float *sqrt_dd;     // sqrt<d|d> of the event (screening margin)
  // outputs
  float4 *tile_part;        // [n_itile * n_etile] (m1, s1, m2, s2) of x = ln(w_i w_e sum_o Lbar)
  float2 *row_part;         // [n_etile][n_int]
  float2 *col_part;         // [n_itile][n_ext]
  float *tile_ml;           // [n_tiles] best ln L^ML in tile
  long long *tile_arg;      // [n_tiles] packed (i, e, o) of it
  int *tile_npass;          // [n_tiles]
  float *lnl_tile;          // optional [n_int][n_ext]
  float *ml_tile;           // optional [n_int][n_ext]
  int *status;
  int gemm_only;
  int n_pol;                // 2: polarisation-resolved bank (row records REC_P, column records F_p F_p')
  int test_stall;           // producer withholds its first stage (failure-path test)
  unsigned long long wait_ns;  // bound of every mbarrier wait
  // screening: a lower bound of <h|h> at every phase per pair, bf16 [n_int][hmin_ld]
  // (slice-relative rows), or null (the screen forms it itself)
  const __nv_bfloat16 *hmin;
  int64_t hmin_ld;
  // screening statistics (null: not counted): [0] pairs that passed the first
  // bound, [1] pairs evaluated over the phase grid
  unsigned long long *n_cand;
};

// Error allowance of a single-pass (one rounding of each operand, unit roundoff u)
// ln L^ML of size ml: the <d|h> components carry a relative error ~u of
// sum_b |h||G| <~ sqrt<h|h> sqrt<d|d>, so ln L^ML = x^2/2 (x = dh / sqrt hh)
// moves by about u (ml + sqrt(2 ml) sqrt<d|d>); margin_k = kappa*u scales it.
__host__ __device__ __forceinline__ float screen_margin(float ml, float margin_k, float sqrt_dd) {
  ml = ml > 0.f ? ml : 0.f;
  return margin_k * (ml + sqrtf(2.f * ml) * sqrt_dd);
}

// Tile order: the extrinsic tiles are swept in bands of `band` tiles; within a
// band every bank tile meets every extrinsic tile of the band before the next
// band starts, so the band's extrinsic operand stays resident in L2 while the
// bank streams through once per band.
__host__ __device__ __forceinline__ void super_tile(int st, int n_itile, int n_etile, int band, int &it, int &et) {
  const int per = n_itile * band;
  const int b = st / per;
  const int w = min(band, n_etile - b * band);
  const int rem = st - b * per;
  it = rem / w;
  et = b * band + rem % w;
}

// ---------------------------------------------------------------------------
// PTX helpers (mbarrier, TMA, tcgen05)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
// One try of a phase wait.  The suspend-time hint (ns) lets the hardware park
// the thread until the phase completes or the hint runs out, instead of the
// warp re-issuing the test.
__device__ __forceinline__ uint32_t mbar_try(uint64_t *b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity), "n"(20000)
      : "memory");
  return ok;
}
// Bounded wait: gives up after limit_ns of wall time, records DEV_E_TIMEOUT
// and returns false.  `abort` (shared) lets one timed-out role stop the others.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, int *status,
                                          volatile int *abort, uint64_t limit_ns = 4000000000ull) {
  if (mbar_try(b, parity)) return true;
  uint64_t t0 = global_ns();
  while (true) {
#pragma unroll 1
    for (int k = 0; k < 32; ++k)
      if (mbar_try(b, parity)) return true;
    if (*abort) return false;
    if (global_ns() - t0 > limit_ns) {
      if (status) atomicCAS(status, 0, DEV_E_TIMEOUT);
      *abort = 1;
      return false;
    }
  }
}
// 3-D tile load: box {x, y, z} lands in shared memory as [z][y][x].
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, "
      "%5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}
__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap *map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(map) : "memory");
}
// K-major operand tile, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc_k128(const void *p) {
  uint64_t a = smem_u32(p);
  return ((a >> 4) & 0x3FFFull) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// Instruction descriptor, kind::f16: D = F32, A/B = bf16 (1) or f16 (0), K-major.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N, bool bf16) {
  return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Approximate reciprocal square root (PTX rsqrt.approx, relative error below
// 2^-22 for normal inputs; subnormal inputs flush to zero).
__device__ __forceinline__ float rsqrt_ftz(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// x rsqrt(x) with x floored at 1e-30: within a few ulp of sqrt(x) for x >= 1e-30
// and above it below, so (1 + 2e-6) times it is never below sqrt(x) (bounds only).
__device__ __forceinline__ float sqrt_near(float x) {
  x = fmaxf(x, 1e-30f);
  return x * rsqrt_ftz(x);
}

// ---------------------------------------------------------------------------
// CTA pairs (a cluster of two CTAs whose MMAs run as one with cta_group::2):
// rank, peer addresses, remote arrivals, the cluster barrier and the pair
// forms of the tcgen05 allocation, MMA and commit.  Every tcgen05 instruction
// of a pair kernel takes cta_group::2.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// shared::cluster address of the variable at shared address `addr` in CTA `rank`
__device__ __forceinline__ uint32_t peer_addr(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc_pair(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_mma_pair(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
      : "memory");
}
// arrives once on the barrier at this shared offset in every CTA of `mask` when
// the pair MMAs issued so far by this thread complete
__device__ __forceinline__ void tc_commit_pair(uint64_t *bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"(mask)
      : "memory");
}
// 3-D tile load into this CTA's shared memory whose completion is counted on
// the barrier at shared::cluster address `bar` (this CTA's or its pair's)
__device__ __forceinline__ void tma_load_3d_pair(void *dst, const CUtensorMap *map, uint32_t bar, int x, int y,
                                                 int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
      "%4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(bar), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// Order-preserving float max for values >= 0.
__device__ __forceinline__ void atomic_max_nonneg(float *addr, float v) {
  atomicMax(reinterpret_cast<int *>(addr), __float_as_int(v));
}

}  // namespace dotpe
