// K3: fused <d|h> GEMM on the 5th-generation tensor cores + marginalisation epilogue.
//
// Persistent kernel, one CTA per SM, warp-specialised:
//   warp 0      TMA producer: bank tile A (128 rows x 2 k-blocks of 64) and
//               extrinsic tile B (64 rows = 32 samples x (re, im), 2 k-blocks)
//               into a ring of stages; each load is one 3-D box spanning two
//               k-blocks (one TMA transaction per operand and stage: the per-CTA
//               TMA rate grows with the transaction size)
//   warp 1      TMEM allocator and tcgen05.mma issuer (one elected lane)
//   warps 2..9  epilogue (two warps per TMEM lane quadrant, each taking half
//               of the tile's extrinsic samples): tcgen05.ld of the accumulators,
//               <h|h> coefficients, phase grid, ML cut, distance marginal,
//               log-sum-exp partials
// Tile = 128 bank rows x TEV extrinsic samples, all modes: accumulators for mode
// m live in TMEM columns [buf * 4 * 2TEV + 2TEV m, +2TEV).  Per mode the GEMM is the
// real-ified complex product of Eq. dh_ieo (K = 2B, padded to a multiple of 64).
// TEV = 32: two buffers, so the epilogue of tile t overlaps the MMAs of tile
// t+1; split precision adds the hi*lo and lo*hi passes into the same
// accumulator.  TEV = 64 (screening pass and GEMM-only runs): one buffer of
// N = 128 per mode fills TMEM, so the epilogue and the next tile's MMAs take
// turns, but every bank byte brought into shared memory feeds twice the MMA
// work (64 instead of 43 flops per operand byte); a work tile then holds the
// partial tiles (it, 2 wt) and (it, 2 wt + 1) of the 32-sample tile grid that
// the outputs are indexed by.  With
// SEP (split only) a tile is taken in two halves of 16 samples (N = 32), each
// with four accumulator sets: hi*hi goes round-robin into three (k16 step t
// into set t mod 3) and the small hi*lo + lo*hi terms into the fourth, all
// added in the epilogue.  The tensor cores' FP32 accumulation truncates at
// every step, with an error that grows with the accumulator's magnitude and
// the number of steps: three interleaved chains of a third of the steps, each
// summing about a third of the value, cut the hi*hi truncation error about
// threefold, and keeping the small terms apart keeps their steps out of the
// large chains.  The cost is the overlap of a half's epilogue with the next
// half's MMAs and a second pass over the bank tile's operand stages.
// A launch may carry a gate: a device word per event; work items of events
// whose word differs from the launch's expected value are skipped by every
// role alike (two variants are launched, each event's word picks the one that
// processes its tiles).
//
// One launch serves a batch of events over one bank (a single event is a batch
// of one): the work items are the events' tiles one event after the other
// (banded order within each), or an (event, tile) list written on the device.
// The epilogue copies an event's parameters into shared memory when its work
// crosses into the next event.
#pragma once
#include "common.cuh"
#include "epilogue.cuh"
#include "kernels.h"

namespace dotpe {

namespace {
constexpr int TI = TC_TI, TE = TC_TE, BK = 64;
constexpr int NEPI = 8;              // epilogue warps
constexpr int NT = (2 + NEPI) * 32;  // 320 threads
constexpr int EPT = NEPI * 32;       // epilogue threads
constexpr uint32_t A_BYTES = TI * BK * 2;  // one k-block of the bank tile
constexpr int KBX = 2;  // k-blocks per stage (one 3-D TMA box)
// Pipeline: single pass = 4 stages of {A, B} x 2 k-blocks (48 KB; 3 x 64 KB
// with the 64-sample tile, 4 x 48 KB when a CTA pair shares it); split
// precision = 2 stages of {A_hi, A_lo, B_hi, B_lo} x 2 k-blocks (96 KB), whose
// three MMA groups (hi*hi, hi*lo, lo*hi) share one load of each plane.
template <bool SPLIT, int TEV, bool PAIR = false> struct Pipe {
  static constexpr int BN = 2 * TEV;  // extrinsic operand rows of a tile: N of every MMA
  static constexpr int NPL = SPLIT ? 2 : 1;
  static constexpr int ST = SPLIT ? 2 : (PAIR ? 4 : (TEV == 64 ? 3 : 4));
  // one k-block of the extrinsic operand in this CTA (a pair: half of the N rows each)
  static constexpr uint32_t B_BYTES = (PAIR ? BN / 2 : BN) * BK * 2;
  static constexpr uint32_t A_ST = KBX * A_BYTES, B_ST = KBX * B_BYTES;  // per plane
  static constexpr uint32_t STAGE = NPL * (A_ST + B_ST);
  static constexpr uint32_t BUF_COLS = MAXM * BN;  // TMEM columns of one accumulator set
};
constexpr uint32_t TMEM_COLS = 512;
static_assert(2 * Pipe<false, 32>::BUF_COLS <= TMEM_COLS && Pipe<false, 64>::BUF_COLS <= TMEM_COLS, "TMEM budget");

// TEV = 32 carries the general epilogue (marginalisation, partial sums through
// shared memory); TEV = 64 only the screening and GEMM-only epilogues.
constexpr int CAND_POOL = 32;  // candidate pairs per epilogue warp and 64-sample tile kept in shared memory
template <int TEV> struct TcTail {
  static constexpr bool GEN = (TEV == 32);
  static constexpr int XS_LD = TEV + 1;
  EpiParams ep;  // parameters of the event whose tile the epilogue is on
  float xs[GEN ? TI * XS_LD : 1];
  alignas(16) float qs[TEV * MAXD * REC];  // read as float4 records
  double lwe[GEN ? TEV : 1];
  float2 ph[7 * MAXPHI];
  float2 rowh[GEN ? TI : 1];  // second-half row partial of each row
  float wm1[NEPI], ws1[NEPI], wm2[NEPI], ws2[NEPI], wml[NEPI];
  // 64-sample screen: per-warp pool of candidate pairs taken out of TMEM
  // (Z_m of every mode, and the owner lane and sample of the pair)
  alignas(16) float pz[TEV == 64 ? NEPI * CAND_POOL * 2 * MAXM : 1];
  int ptag[TEV == 64 ? NEPI * CAND_POOL : 1];
  long long warg[NEPI];
  int wnp[NEPI];
  uint64_t full[4], empty[4], tfull[2], tempty[2], drain;
  uint64_t mfull;  // 64-sample tiles: the accumulators of modes 0 and 1 are complete
  uint32_t tmem_slot;
  int abort_flag;
};
template <bool SPLIT, int TEV, bool PAIR = false>
constexpr size_t smem_bytes() {
  return 1024 + (size_t)Pipe<SPLIT, TEV, PAIR>::ST * Pipe<SPLIT, TEV, PAIR>::STAGE + sizeof(TcTail<TEV>);
}
static_assert(smem_bytes<true, 32>() <= 232448 && smem_bytes<false, 32>() <= 232448 &&
                  smem_bytes<false, 64>() <= 232448 && smem_bytes<false, 64, true>() <= 232448,
              "shared memory budget");
}  // namespace

// 32 lanes x 32-bit, 2 consecutive columns per thread.
__device__ __forceinline__ void tmem_ld2(uint32_t taddr, float &a, float &b) {
  uint32_t r0, r1;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(taddr));
  a = __uint_as_float(r0);
  b = __uint_as_float(r1);
}

// An upper bound of sqrt(x) for x >= 0 from the approximate reciprocal square
// root (a few ulp; the factor covers it): bounds only, never values.
__device__ __forceinline__ float sqrt_up(float x) {
  return x > 0.f ? x * rsqrtf(x) * 1.000002f : 0.f;
}

// 32 lanes x 32-bit, 16 consecutive columns per thread (column a multiple of 16).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// Work item w -> (event k, tile it, et): entry w of the device list, or the
// event whose range [begin[k], begin[k+1]) holds w and, within it, the banded
// order of super_tile.
// With TEV = 64 the grid-mode items are 64-sample work tiles (et counts them):
// ceil(n_etile / 2) per bank tile, banded in half as many of them.
// PAIR: the item is a 256-row pair tile; CTA `rank` of the pair takes its bank tile 2 it + rank.
// Returns false for a band-order item that a pilot tile has already screened
// (every role of the kernel skips it: the pilot pass wrote all its outputs,
// with a threshold no higher than the band-order pass would use).
template <int NB, int TEV, bool PAIR = false>
__device__ __forceinline__ bool work_tile(const TcBatch<NB> &Bt, int w, int &k, int &it, int &et,
                                          uint32_t rank = 0) {
  constexpr int RS = TEV / TE;  // 32-sample tiles per work tile
  if (Bt.glist) {
    const int2 q = Bt.glist[w];
    k = q.x;
    it = q.y / Bt.w[k].n_etile;
    et = q.y - it * Bt.w[k].n_etile;
    return true;
  }
  k = 0;
  if (NB > 1) {
    int lo = 0, hi = Bt.n - 1;  // largest k with begin[k] <= w
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (Bt.begin[mid] <= w) lo = mid;
      else hi = mid - 1;
    }
    k = lo;
  }
  const TcEvent &W = Bt.w[k];
  const int ni = PAIR ? (W.n_itile + 1) / 2 : W.n_itile;  // bank tiles (pair tiles) of the event
  const int nw = (W.n_etile + RS - 1) / RS, bw = W.band / RS;
  const int np = tc_pilot_tiles(W, TEV, PAIR);
  const int local = w - Bt.begin[k];
  const int nc = min(nw, TC_PILOT_COLS), nr = (np + nc - 1) / nc;
  bool run = true;
  if (local < np) {
    // pilot tile: row a of the grid of spread bank tiles, column c of the spread extrinsic tiles
    const int a = local / nc, c = local - a * nc;
    it = (int)(((long long)a * ni) / nr);
    et = (int)(((2ll * c + 1) * nw) / (2 * nc));
  } else {
    super_tile(local - np, ni, nw, bw < 1 ? 1 : (bw > nw ? nw : bw), it, et);
    if (np > 0) {
      // a pilot tile again: the (a, c) of the grid that maps to (it, et), if any
      // (column spacing nw / nc >= 1 and row spacing ni / nr >= 1: at most one)
      const int c0 = et * nc / nw;  // et < nw, nc <= TC_PILOT_COLS: no overflow
      for (int c = max(0, c0 - 1); c <= min(nc - 1, c0 + 1); ++c)
        if ((2 * c + 1) * nw / (2 * nc) == et) {
          const int a0 = (int)(((long long)it * nr) / ni);
          for (int a = max(0, a0 - 1); a <= a0 + 1; ++a)
            if (a < nr && (int)(((long long)a * ni) / nr) == it && a * nc + c < np) run = false;
        }
    }
  }
  if (PAIR) it = 2 * it + (int)rank;
  return run;
}

// PAIR: launched in clusters of two CTAs that run each MMA as one (cta_group::2,
// M = 256): each CTA loads its own 128 bank rows and half of the tile's N
// extrinsic rows, the even CTA issues the MMAs and commits them to both, and
// each CTA's epilogue reads its own rows' accumulators from its own TMEM.
template <bool BF16, int HH, bool SPLIT, int NB, bool SEP, int TEV, bool PAIR = false>
__global__ void __launch_bounds__(NT, 1)
    tc_fused_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ TcBatch<NB> Bt,
                    const TcCommon C) {
  static_assert(SPLIT || !SEP, "a separate low-order accumulator needs split operands");
  static_assert(TEV == 32 || (TEV == 64 && !SPLIT && HH != 2), "64-sample tiles: single-pass mode banks");
  static_assert(!PAIR || (TEV == 64 && NB == 1), "CTA pairs: 64-sample tiles of one event");
  using PP = Pipe<SPLIT, TEV, PAIR>;
  using TcTail = dotpe::TcTail<TEV>;
  constexpr int ST = PP::ST, NPL = PP::NPL, BN = PP::BN;
  constexpr uint32_t STAGE_BYTES = PP::STAGE, A_ST = PP::A_ST, B_ST = PP::B_ST, B_BYTES = PP::B_BYTES;
  constexpr uint32_t BUF_COLS = PP::BUF_COLS;
  constexpr int EHALF = TEV / 2;  // extrinsic samples per epilogue thread and tile
  constexpr int XS_LD = TcTail::XS_LD;
  constexpr bool ONEBUF = SEP || TEV == 64;  // one accumulator set in flight
  constexpr int NUSE = SEP ? 2 : 1;           // accumulator uses per work tile (SEP: two 16-sample halves)
  constexpr int SEP_N = BN / 2;               // SEP: N of each MMA (one half's B rows)
  constexpr uint32_t SEP_SET = 128;           // SEP: TMEM columns of one accumulator set (4 modes x N)
  static_assert(!SEP || (TEV == 32 && 4 * SEP_SET <= TMEM_COLS), "SEP accumulator sets");
  extern __shared__ uint8_t smem_raw[];
  uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // stage s, plane p: A at sA + (s NPL + p) A_ST as [KBX][128 rows][64],
  //                   B at sB + (s NPL + p) B_ST as [KBX][64 rows][64]
  uint8_t *sA = base;
  uint8_t *sB = base + ST * NPL * A_ST;
  TcTail &T = *reinterpret_cast<TcTail *>(base + (size_t)ST * STAGE_BYTES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int M = C.n_modes;
  const int n_work = Bt.glist ? *Bt.glist_n : Bt.begin[Bt.n];
  const int nst = (C.kb + KBX - 1) / KBX;  // stages per mode (an odd last k-block is zero-filled)
  const unsigned long long wait_ns = Bt.w[0].P.wait_ns;
  // work items: per CTA, or per CTA pair (consecutive blocks form a cluster)
  const uint32_t rank = PAIR ? cluster_rank() : 0u;
  const int w0 = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
  const int wstep = PAIR ? (int)(gridDim.x >> 1) : (int)gridDim.x;
  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(&T.full[s], 1);
      mbar_init(&T.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&T.tfull[b], 1);
      mbar_init(&T.tempty[b], PAIR ? 2 * NEPI : NEPI);  // a pair: both CTAs' epilogue warps
    }
    mbar_init(&T.drain, 1);
    mbar_init(&T.mfull, 1);
    T.abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == 0 && lane == 0) {
    tma_prefetch_desc(&mapA);
    tma_prefetch_desc(&Bt.mapB[0]);
  }
  if (warp == 1) {
    if constexpr (PAIR) tmem_alloc_pair(&T.tmem_slot, TMEM_COLS);
    else tmem_alloc(&T.tmem_slot, TMEM_COLS);
  }
  tc_fence_before();
  __syncthreads();
  // a pair: the peer's barriers are initialised before any copy or arrival reaches them
  if constexpr (PAIR) cluster_sync_all();
  tc_fence_after();
  const uint32_t tmem = T.tmem_slot;
  volatile int *abortp = &T.abort_flag;
  // this CTA's epilogue warps hand the accumulator set back (a pair: to the even CTA's barrier)
  auto release_acc = [&](int b) {
    if (PAIR && rank != 0) mbar_arrive_remote(peer_addr(smem_u32(&T.tempty[b]), 0));
    else mbar_arrive(&T.tempty[b]);
  };

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      uint32_t q = 0;
      bool ok = !Bt.w[0].P.test_stall;
      for (int w = w0; w < n_work && ok; w += wstep) {
        int k, it, et;
        if (!work_tile<NB, TEV, PAIR>(Bt, w, k, it, et, rank)) continue;
        if (Bt.gate && Bt.gate[k] != Bt.gate_want) continue;
        const TcEvent &W = Bt.w[k];
        for (int h2 = 0; h2 < NUSE; ++h2)
        for (int m = 0; m < M && ok; ++m) {
          const int arow = m * C.a_mode_rows + W.a_row0 + it * TI;
          // a pair: this CTA's half of the tile's extrinsic rows
          const int brow = m * W.b_mode_rows + et * BN + (PAIR ? (int)rank * (BN / 2) : 0);
          for (int ks = 0; ks < nst; ++ks, ++q) {
            const int s = q % ST;
            const uint32_t n = q / ST;
            if (n > 0 && !(ok = mbar_wait(&T.empty[s], (n - 1) & 1, nullptr, abortp, wait_ns))) break;
            if constexpr (PAIR) {
              // both CTAs' copies complete on the even CTA's barrier, which expects them all
              if (rank == 0) mbar_expect_tx(&T.full[s], 2 * STAGE_BYTES);
              const uint32_t fb = peer_addr(smem_u32(&T.full[s]), 0);
              tma_load_3d_pair(sA + s * A_ST, &mapA, fb, 0, arow, ks * KBX);
              tma_load_3d_pair(sB + s * B_ST, &Bt.mapB[k], fb, 0, brow, ks * KBX);
            } else {
              mbar_expect_tx(&T.full[s], STAGE_BYTES);
#pragma unroll
              for (int pl = 0; pl < NPL; ++pl) {
                tma_load_3d(sA + (s * NPL + pl) * A_ST, &mapA, &T.full[s], 0, pl * C.a_plane_rows + arow, ks * KBX);
                tma_load_3d(sB + (s * NPL + pl) * B_ST, &Bt.mapB[k], &T.full[s], 0, pl * W.b_plane_rows + brow,
                            ks * KBX);
              }
            }
          }
        }
      }
      if (PAIR && rank != 0 && !ok) {
        // the odd CTA's copies complete on the even CTA's barrier: give those in flight time to land
        const uint64_t t0 = global_ns();
        while (global_ns() - t0 < 2000000ull) {
        }
      } else if (!ok) {
        // let copies already in flight land before the CTA exits
        uint32_t first = q > (uint32_t)ST ? q - ST : 0;
        for (uint32_t j = first; j < q; ++j) {
          volatile int no_abort = 0;
          mbar_wait(&T.full[j % ST], (j / ST) & 1, nullptr, &no_abort, 200000000ull);
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    // The whole warp walks the schedule (so descriptors and addresses stay
    // warp-uniform); lane 0 issues every MMA and commit (a commit tracks the
    // MMAs of the thread that issues it).
    // (a pair: the even CTA issues M = 256 MMAs over both CTAs' operands; the
    // odd CTA's MMA warp only holds its TMEM until they are done)
    constexpr uint32_t idesc = idesc_f16(PAIR ? 256 : 128, BN, BF16);
    const bool issuer = (lane == 0);
    uint32_t q = 0, u = 0;
    bool ok = !(PAIR && rank != 0);
    for (int w = w0; w < n_work && ok; w += wstep) {
      {
        int k, it, et;
        if (!work_tile<NB, TEV, PAIR>(Bt, w, k, it, et, rank)) continue;
        if (Bt.gate && Bt.gate[k] != Bt.gate_want) continue;
      }
      for (int h2 = 0; h2 < NUSE && ok; ++h2) {
      const int b = ONEBUF ? 0 : (u & 1);
      const uint32_t use = ONEBUF ? u : (u >> 1);
      ++u;
      if (use > 0) ok = __all_sync(0xffffffffu, mbar_wait(&T.tempty[b], (use - 1) & 1, nullptr, abortp, wait_ns));
      if (!ok) break;
      tc_fence_after();
      for (int m = 0; m < M && ok; ++m) {
        const uint32_t dcol = tmem + b * BUF_COLS + m * BN;
        const uint32_t dlo = tmem + 3 * SEP_SET + m * SEP_N;  // SEP: the hi*lo + lo*hi accumulator
        for (int ks = 0; ks < nst; ++ks, ++q) {
          const int s = q % ST;
          const uint32_t n = q / ST;
          ok = __all_sync(0xffffffffu, mbar_wait(&T.full[s], n & 1, nullptr, abortp, wait_ns));
          if (!ok) break;
          tc_fence_after();
          if (issuer) {
#pragma unroll
            for (int kx = 0; kx < KBX; ++kx) {
              const uint64_t ah = sdesc_k128(sA + (s * NPL) * A_ST + kx * A_BYTES);
              const uint64_t al = sdesc_k128(sA + (s * NPL + NPL - 1) * A_ST + kx * A_BYTES);
              // SEP: this half's 32 B rows (8-row groups of 1024 bytes)
              const uint32_t boff = SEP ? (uint32_t)h2 * SEP_N * 128u : 0u;
              const uint64_t bh = sdesc_k128(sB + (s * NPL) * B_ST + kx * B_BYTES + boff);
              const uint64_t bl = sdesc_k128(sB + (s * NPL + NPL - 1) * B_ST + kx * B_BYTES + boff);
#pragma unroll
              for (int k = 0; k < BK / 16; ++k) {
                if (SEP) {
                  constexpr uint32_t idesc_sep = idesc_f16(128, SEP_N, BF16);
                  const int t16 = (ks * KBX + kx) * (BK / 16) + k;  // k16 step of this mode's chain
                  const uint32_t dhh = tmem + (uint32_t)(t16 % 3) * SEP_SET + m * SEP_N;
                  tc_mma(dhh, ah + 2 * k, bh + 2 * k, idesc_sep, t16 >= 3 ? 1u : 0u);      // hi * hi
                  tc_mma(dlo, ah + 2 * k, bl + 2 * k, idesc_sep, t16 > 0 ? 1u : 0u);       // hi * lo
                  tc_mma(dlo, al + 2 * k, bh + 2 * k, idesc_sep, 1u);                      // lo * hi
                } else if (PAIR) {
                  tc_mma_pair(dcol, ah + 2 * k, bh + 2 * k, idesc, (ks | kx | k) ? 1u : 0u);
                } else {
                  tc_mma(dcol, ah + 2 * k, bh + 2 * k, idesc, (ks | kx | k) ? 1u : 0u);
                  if (SPLIT) {
                    tc_mma(dcol, ah + 2 * k, bl + 2 * k, idesc, 1u);  // hi * lo
                    tc_mma(dcol, al + 2 * k, bh + 2 * k, idesc, 1u);  // lo * hi
                  }
                }
              }
            }
            if (PAIR) tc_commit_pair(&T.empty[s], 0x3);
            else tc_commit(&T.empty[s]);
          }
          __syncwarp();
        }
        if (TEV == 64 && m == 1 && M >= 3 && ok && issuer) {
          // modes 0 and 1 are issued (the MMAs run mode after mode): the screen's
          // epilogue reads them while the other modes' MMAs run
          if (PAIR) tc_commit_pair(&T.mfull, 0x3);
          else tc_commit(&T.mfull);
        }
        __syncwarp();
      }
      if (ok && issuer) {
        if (PAIR) tc_commit_pair(&T.tfull[b], 0x3);
        else tc_commit(&T.tfull[b]);
      }
      __syncwarp();
      }
    }
    // all MMAs of this CTA (a pair: of the even CTA, on both) complete before TMEM is released
    volatile int no_abort = 0;
    if (PAIR && rank != 0) {
      // the even CTA commits the drain once its work is issued: wait for it over the whole launch
      mbar_wait(&T.drain, 0, nullptr, &no_abort, 20000000000ull);
    } else {
      if (issuer) {
        if (PAIR) tc_commit_pair(&T.drain, 0x3);
        else tc_commit(&T.drain);
      }
      __syncwarp();
      mbar_wait(&T.drain, 0, nullptr, &no_abort, 500000000ull);
    }
  } else {
    // ---------------- epilogue (256 threads: one tile row, half the samples each) ----------------
    const int ew = warp - 2;      // 0..7
    const int quad = warp & 3;    // TMEM lane quadrant this warp may access
    const int half = ew >> 2;     // which 16 of the tile's 32 extrinsic samples
    const int row = quad * 32 + lane;
    const int etid = threadIdx.x - 64;
    // one event: its parameters straight from kernel-parameter space (constant
    // bank); a batch: the current event's copy in shared memory
    const EpiParams &P = (NB == 1) ? Bt.w[0].P : T.ep;
    bool store = false;
    float zs = 1.f;
    constexpr int NREC = (HH == 2) ? POL_TC_MAXD * REC_POL : MAXD * REC;  // row record floats in registers
    float mrec[NREC];

    double lwi = 0.0;
    int cur_it = -1, cur_k = -1;
    uint32_t u = 0;
    for (int w = w0; w < n_work; w += wstep) {
      int k, it, et;
      if (!work_tile<NB, TEV, PAIR>(Bt, w, k, it, et, rank)) continue;
      if (Bt.gate && Bt.gate[k] != Bt.gate_want) continue;
      const int b = ONEBUF ? 0 : (u & 1);
      const uint32_t use = ONEBUF ? u : (u >> 1);
      u += NUSE;
      if (k != cur_k) {
        // the next event: its parameters and phase tables into shared memory
        named_bar_sync(1, EPT);
        {
          const int *src = reinterpret_cast<const int *>(&Bt.w[k].P);
          int *dst = reinterpret_cast<int *>(&T.ep);
          for (int q = etid; q < (int)(sizeof(EpiParams) / 4); q += EPT) dst[q] = src[q];
        }
        named_bar_sync(1, EPT);
        fill_phase_tables(T.ph, P, etid, EPT);
        store = (P.lnl_tile != nullptr);
        zs = P.z_scale / (P.g_scale ? *P.g_scale : 1.f);
        cur_k = k;
        cur_it = -1;
      }
      const bool etv = true;
      const int t = it * Bt.w[k].n_etile + et;
      const int64_t i = (int64_t)it * TI + row;
      const bool vi = i < P.n_int;
      const int64_t e0 = (int64_t)et * TEV;
      // the row record of this thread's bank row into registers (64-sample tiles:
      // only where it is used, so that it holds no registers through pass 1)
      auto load_mrec = [&]() {
#pragma unroll
        for (int k = 0; k < NREC; ++k) mrec[k] = 0.f;
        if constexpr (HH == 2) {
          // row records of REC_P floats per detector, the first REC_POL kept
          const float4 *src = reinterpret_cast<const float4 *>(P.mx + i * P.n_det * REC_P);
#pragma unroll
          for (int d = 0; d < POL_TC_MAXD; ++d)
#pragma unroll
            for (int v = 0; v < REC_P / 4; ++v) {
              if (vi && d < P.n_det) {
                const float4 x = __ldg(src + d * (REC_P / 4) + v);
                const float xs4[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int c = 0; c < 4; ++c)
                  if (4 * v + c < REC_POL) mrec[d * REC_POL + 4 * v + c] = xs4[c];
              }
            }
        } else {
          const float4 *src = reinterpret_cast<const float4 *>(P.mx + i * P.n_det * REC);
#pragma unroll
          for (int k = 0; k < MAXD * REC / 4; ++k) {
            if (vi && k < P.n_det * REC / 4) {
              float4 v = __ldg(src + k);
              mrec[4 * k] = v.x; mrec[4 * k + 1] = v.y; mrec[4 * k + 2] = v.z; mrec[4 * k + 3] = v.w;
            }
          }
        }
      };
      if (it != cur_it) {
        if constexpr (TEV == 32) load_mrec();
        lwi = (vi && P.lw_int) ? P.lw_int[i] : 0.0;
        cur_it = it;
      }
      // column records of the tile's samples, a float4 at a time (compile-time
      // divisors; detectors beyond n_det are never read)
      for (int f = etid; f < TEV * MAXD * (REC / 4); f += EPT) {
        const int e = f / (MAXD * (REC / 4)), r = f % (MAXD * (REC / 4)), d = r / (REC / 4), v = r % (REC / 4);
        if (d < P.n_det) {
          float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
          if (e0 + e < P.n_ext)
            x = __ldg(reinterpret_cast<const float4 *>(P.qx + ((e0 + e) * P.n_det + d) * REC) + v);
          *reinterpret_cast<float4 *>(&T.qs[(e * MAXD + d) * REC + 4 * v]) = x;
        }
      }
      if constexpr (TcTail::GEN)
        for (int k = etid; k < TEV; k += EPT) T.lwe[k] = (P.lw_ext && e0 + k < P.n_ext) ? P.lw_ext[e0 + k] : 0.0;
      named_bar_sync(1, EPT);
      float thr = tile_threshold(P);
      // 64-sample screen: for each of the thread's pairs the lower bound of
      // <h|h> at every phase that pair_bound uses, C_0 - 2 sum_delta |C_delta|
      // (Eq. hh_ieo), formed while the MMAs of the tile run
      // (a rolled loop into a per-thread array that lives in local memory: small
      // code, no register pressure, read back once per pair in pass 1)
      float hl[TEV == 64 ? TEV / 2 : 1];
      if constexpr (TEV == 64) {
        if (!P.gemm_only && P.hmin) {
          // the bound from the tensor-core <h|h> pass (bf16, rounded down)
          const int64_t ib = vi ? i : 0;
          const uint4 *src = reinterpret_cast<const uint4 *>(P.hmin + ib * P.hmin_ld + e0 + half * EHALF);
#pragma unroll
          for (int v4 = 0; v4 < EHALF / 8; ++v4) {
            const uint4 w = __ldcs(src + v4);  // read once: evict first, keep the operand band in L2
            const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              hl[8 * v4 + 2 * c] = __uint_as_float(ws[c] << 16);
              hl[8 * v4 + 2 * c + 1] = __uint_as_float(ws[c] & 0xffff0000u);
            }
          }
        } else if (!P.gemm_only) {
          load_mrec();
#pragma unroll 1
          for (int j = 0; j < EHALF; ++j) {
            float C0, Cr[3], Ci[3];
            hh_tile<HH>(mrec, &T.qs[(half * EHALF + j) * MAXD * REC], P, C0, Cr, Ci);
            float h = C0;
#pragma unroll
            for (int q = 0; q < 3; ++q) h -= 2.f * sqrt_up(Cr[q] * Cr[q] + Ci[q] * Ci[q]);
            hl[j] = h;
          }
        }
      }
      // 64-sample screen with three or four modes: modes 0 and 1 complete first;
      // their share of sum_m |Z_m| per pair is read while the other modes' MMAs run
      const bool early = TEV == 64 && !P.gemm_only && M >= 3;
      float a01[TEV == 64 ? EHALF : 1];
      if constexpr (TEV == 64) {
        if (early) {
          if (!mbar_wait(&T.mfull, use & 1, nullptr, abortp, wait_ns)) break;
          tc_fence_after();
          const uint32_t tb = tmem + ((uint32_t)(quad * 32) << 16);
#pragma unroll
          for (int g = 0; g < EHALF / 8; ++g) {
            float v[2][16];
#pragma unroll
            for (int m = 0; m < 2; ++m) tmem_ld16(tb + m * BN + 2 * (half * EHALF + 8 * g), v[m]);
            tmem_ld_wait();
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              float s = 0.f;
#pragma unroll
              for (int m = 0; m < 2; ++m) s += sqrt_near(fmaf(v[m][2 * q], v[m][2 * q], v[m][2 * q + 1] * v[m][2 * q + 1]));
              a01[8 * g + q] = s;
            }
          }
        }
      }
      if (!mbar_wait(&T.tfull[b], use & 1, nullptr, abortp, wait_ns)) break;
      tc_fence_after();

      if constexpr (TEV == 64) {
        // ---- 64-sample work tile: screening (or GEMM-only) of partial tiles 2 et + half ----
        const int n_etile = Bt.w[k].n_etile;
        const int pe = 2 * et + half;  // this thread's 32-sample partial tile
        const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16);
        float best = -1.f;
        long long barg = 0x7fffffffffffffffLL;
        if (P.gemm_only) {
          // the accumulators summed (keeps every TMEM read; the result is not valid)
          float sx = 0.f;
#pragma unroll
          for (int g = 0; g < EHALF / 8; ++g)
#pragma unroll
            for (int m = 0; m < MAXM; ++m)
              if (m < M) {
                float v[16];
                tmem_ld16(tbase + m * BN + 2 * (half * EHALF + 8 * g), v);
                tmem_ld_wait();
#pragma unroll
                for (int q = 0; q < 16; ++q) sx += v[q];
              }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) release_acc(0);
          best = (vi && sx == sx) ? fabsf(sx) : -1.f;
        } else {
          // Pass 1 (the accumulators read 16 columns at a time): the bound of
          // pair_bound, (sum_m |Z_m|)^2 / (2 hl), against the threshold; the
          // pairs that reach it are the candidates.  Each candidate's Z_m go to
          // the warp's pool in shared memory as soon as its group of 8 samples is
          // tested, so the buffer can be released before any candidate is
          // evaluated; candidates beyond the pool stay in `cand`.
          // (the sum of sqrt_near is within a factor 1 + 2e-6 of the sum of |Z_m|)
          const float cm = zs * zs * 1.000006f;
          const float thr2 = 2.f * thr;
          uint32_t cand = 0;
          int npool = 0;  // warp-uniform
          int ncand = 0;  // the warp's candidates (warp-uniform)
          int neval = 0;  // this lane's evaluations over the phase grid
          float *pz = &T.pz[ew * CAND_POOL * 2 * MAXM];
          int *ptag = &T.ptag[ew * CAND_POOL];
          const int mlast = M > 2 ? 2 : 0;  // first mode of the pair left in v after the mode loop
#pragma unroll
          for (int g = 0; g < EHALF / 8; ++g) {
            float a[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) a[q] = early ? a01[8 * g + q] : 0.f;
            float v[2][16];
#pragma unroll
            for (int m0 = 0; m0 < MAXM; m0 += 2) {
              if (early && m0 == 0) continue;  // modes 0 and 1 are in a01
              // two modes per wait
#pragma unroll
              for (int m = m0; m < m0 + 2; ++m)
                if (m < M) tmem_ld16(tbase + m * BN + 2 * (half * EHALF + 8 * g), v[m - m0]);
              tmem_ld_wait();
#pragma unroll
              for (int m = m0; m < m0 + 2; ++m)
                if (m < M) {
#pragma unroll
                  for (int q = 0; q < 8; ++q)
                    a[q] += sqrt_near(fmaf(v[m - m0][2 * q], v[m - m0][2 * q], v[m - m0][2 * q + 1] * v[m - m0][2 * q + 1]));
                }
            }
            uint32_t gc = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const int j = 8 * g + q;
              const bool valid = vi && (e0 + half * EHALF + j < P.n_ext);
              const bool reject = hl[j] > 0.f && cm * a[q] * a[q] < thr2 * hl[j];
              if (valid && !reject) gc |= 1u << q;
            }
            if (__any_sync(0xffffffffu, gc != 0u)) {
              // pool slots: exclusive prefix of the lanes' candidate counts
              const int cnt = __popc(gc);
              int incl = cnt;
#pragma unroll
              for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
              }
              const int total = __shfl_sync(0xffffffffu, incl, 31);
              ncand += total;
              int slot = npool + incl - cnt;
              uint32_t kept = 0;
#pragma unroll
              for (int q = 0; q < 8; ++q)
                if ((gc >> q) & 1u) {
                  if (slot < CAND_POOL) {
                    ptag[slot] = (lane << 8) | (half * EHALF + 8 * g + q);
#pragma unroll
                    for (int m = 0; m < 2; ++m)
                      if (mlast + m < M)
                        *reinterpret_cast<float2 *>(&pz[slot * 2 * MAXM + 2 * (mlast + m)]) =
                            make_float2(v[m][2 * q], v[m][2 * q + 1]);
                    kept |= 1u << q;
                  } else {
                    cand |= 1u << (8 * g + q);
                  }
                  ++slot;
                }
              if (mlast > 0) {
                // modes 0 and 1 of the group once more
#pragma unroll
                for (int m = 0; m < 2; ++m) tmem_ld16(tbase + m * BN + 2 * (half * EHALF + 8 * g), v[m]);
                tmem_ld_wait();
                int sl = npool + incl - cnt;
#pragma unroll
                for (int q = 0; q < 8; ++q)
                  if ((kept >> q) & 1u) {
#pragma unroll
                    for (int m = 0; m < 2; ++m)
                      *reinterpret_cast<float2 *>(&pz[sl * 2 * MAXM + 2 * m]) = make_float2(v[m][2 * q], v[m][2 * q + 1]);
                    ++sl;
                  }
              }
              npool = min(CAND_POOL, npool + total);
            }
          }
          // Pass 2: the pool, one candidate per lane at a time (the owner's row
          // record read through the cache): the phase grid where the pair's bound still
          // reaches the threshold and the thread's best.  While candidates remain
          // in TMEM beyond the pool, the buffer is kept and the pool refilled
          // from it (the warp takes the lowest pending sample of its lanes at a
          // time); after the last refill the buffer goes back to the MMA warp
          // and the pool is evaluated while the next tile's MMAs run.  The
          // threshold follows the running maximum, raised by every pair
          // evaluated here (a lower bound of the final threshold throughout).
          float pushed = 0.f;
          bool held = true;
#pragma unroll 1
          while (true) {
            const bool more = __any_sync(0xffffffffu, cand != 0u);
            if (!more && held) {
              // the accumulators are no longer needed: release the buffer to the MMA warp
              tc_fence_before();
              __syncwarp();
              if (lane == 0) release_acc(0);
              held = false;
            }
#pragma unroll 1
            for (int k0 = 0; k0 < npool; k0 += 32) {
              const int kk = k0 + lane;
              const bool act = kk < npool;
              const int tag = act ? ptag[kk] : (lane << 8);
              const int owner = tag >> 8, el = tag & 255;
              if (act) {
                const int64_t io = (int64_t)it * TI + quad * 32 + owner;
                const float *mrow = P.mx + io * P.n_det * REC;
                float C0, Cr[3], Ci[3];
                hh_coeffs_by<HH == 1>([&](int q) { return __ldg(mrow + q); }, &T.qs[el * MAXD * REC], P, C0, Cr, Ci);
                float Zr[MAXM], Zi[MAXM];
#pragma unroll
                for (int m = 0; m < MAXM; ++m) {
                  if (m < M) {
                    const float2 z = *reinterpret_cast<const float2 *>(&pz[kk * 2 * MAXM + 2 * m]);
                    Zr[m] = z.x * zs;
                    Zi[m] = z.y * zs;
                  } else {
                    Zr[m] = 0.f;
                    Zi[m] = 0.f;
                  }
                }
                const float bound = pair_bound(Zr, Zi, C0, Cr, Ci);
                if (bound >= thr && !(bound < best)) {
                  int argo;
                  const float ml = pair_ml(Zr, Zi, C0, Cr, Ci, thr, false, P, T.ph, argo);
                  ++neval;
                  const long long gidx = (io * P.n_ext + e0 + el) * (long long)P.n_phi + argo;
                  if (ml > best || (ml == best && gidx < barg)) {
                    best = ml;
                    barg = gidx;
                  }
                  if (P.track_max && ml > pushed && ml > 0.f) {
                    atomic_max_nonneg(P.ml_running, ml);
                    pushed = ml;
                  }
                }
              }
              thr = fmaxf(thr, tile_threshold(P));
            }
            __syncwarp();
            npool = 0;
            if (!more) break;
#pragma unroll 1
            while (npool < CAND_POOL && __any_sync(0xffffffffu, cand != 0u)) {
              const int jl = cand ? (__ffs(cand) - 1) : EHALF;
              const int j = __reduce_min_sync(0xffffffffu, jl);
              const bool mine = ((cand >> j) & 1u) != 0u;
              float zr[MAXM], zi[MAXM];
#pragma unroll
              for (int m = 0; m < MAXM; ++m) {
                if (m < M) tmem_ld2(tbase + m * BN + 2 * (half * EHALF + j), zr[m], zi[m]);
                else { zr[m] = 0.f; zi[m] = 0.f; }
              }
              tmem_ld_wait();
              const uint32_t bal = __ballot_sync(0xffffffffu, mine);
              const int slot = npool + __popc(bal & ((1u << lane) - 1u));
              if (mine && slot < CAND_POOL) {
                ptag[slot] = (lane << 8) | (half * EHALF + j);
#pragma unroll
                for (int m = 0; m < MAXM; ++m)
                  *reinterpret_cast<float2 *>(&pz[slot * 2 * MAXM + 2 * m]) = make_float2(zr[m], zi[m]);
                cand &= ~(1u << j);
              }
              npool = min(CAND_POOL, npool + __popc(bal));
            }
            __syncwarp();
          }
          if (P.n_cand) {
            const int ne = __reduce_add_sync(0xffffffffu, neval);
            if (lane == 0 && ncand > 0) {
              atomicAdd(&P.n_cand[0], (unsigned long long)ncand);
              atomicAdd(&P.n_cand[1], (unsigned long long)ne);
            }
          }
        }
        // outputs of the two partial tiles: empty marginal partials and each one's best ln L^ML
        warp_argmax(best, barg);
        if (lane == 0) {
          T.wml[ew] = best;
          T.warg[ew] = barg;
        }
        // (a pair's odd CTA past the last bank tile has no outputs: all its rows are invalid)
        const bool tv = it < Bt.w[k].n_itile;
        if (vi && pe < n_etile) P.row_part[(int64_t)pe * P.n_int + i] = make_float2(-INFINITY, 0.f);
        if (tv && etid < TEV && e0 + etid < P.n_ext)
          P.col_part[(int64_t)it * P.n_ext + e0 + etid] = make_float2(-INFINITY, 0.f);
        named_bar_sync(1, EPT);
        if (tv && etid < 2 && 2 * et + etid < n_etile) {
          // warps 4 h .. 4 h + 3 hold partial tile 2 et + h
          float bv = -1.f;
          long long bi = 0x7fffffffffffffffLL;
          for (int q = 4 * etid; q < 4 * etid + 4; ++q)
            if (T.wml[q] > bv || (T.wml[q] == bv && T.warg[q] < bi)) { bv = T.wml[q]; bi = T.warg[q]; }
          const int tp = it * n_etile + 2 * et + etid;
          P.tile_part[tp] = make_float4(-INFINITY, 0.f, -INFINITY, 0.f);
          P.tile_ml[tp] = bv;
          P.tile_arg[tp] = bi;
          P.tile_npass[tp] = 0;
          if (bv > 0.f && P.track_max && !P.gemm_only) atomic_max_nonneg(P.ml_running, bv);
        }
        // the next tile's barrier (after its column records) orders these reads
        // of T.wml before any thread writes it again
        continue;
      } else {

      Lse ra, rb;
      ra.init();
      rb.init();
      float best = -1.f;
      long long barg = 0x7fffffffffffffffLL;
      int np = 0;
      const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + b * BUF_COLS;
      if (!SPLIT && P.screen_ml && !store && !P.gemm_only) {
        // Screening without stored values needs only the tile's best ln L^ML.
        // Pass 1 bounds every pair of this thread (bounds kept in the thread's
        // own xs entries); pass 2 evaluates pairs in decreasing bound order
        // until the next bound lies below both the threshold and the best so far.
        float *xb = &T.xs[row * XS_LD + half * EHALF];
#pragma unroll 1
        for (int j = 0; j < EHALF; ++j) {
          const int64_t e = e0 + half * EHALF + j;
          float Zr[MAXM], Zi[MAXM];
#pragma unroll
          for (int m = 0; m < MAXM; ++m) {
            if (m < M) tmem_ld2(tbase + m * BN + 2 * (half * EHALF + j), Zr[m], Zi[m]);
            else { Zr[m] = 0.f; Zi[m] = 0.f; }
          }
          tmem_ld_wait();
          float bound = -INFINITY;
          if (vi && e < P.n_ext) {
#pragma unroll
            for (int m = 0; m < MAXM; ++m) {
              Zr[m] *= zs;
              Zi[m] *= zs;
            }
            float C0, Cr[3], Ci[3];
            hh_tile<HH>(mrec, &T.qs[(half * EHALF + j) * MAXD * REC], P, C0, Cr, Ci);
            bound = pair_bound(Zr, Zi, C0, Cr, Ci);
          }
          xb[j] = bound;
        }
        // Rounds: each lane picks its highest remaining bound; the warp reads the
        // accumulator columns its lanes picked (tcgen05.ld takes one column for the
        // whole warp), then each lane evaluates its own pick.
        int neval = 0;
#pragma unroll 1
        while (true) {
          int jm = 0;
          float bm = xb[0];
#pragma unroll
          for (int j = 1; j < EHALF; ++j) {
            const float v = xb[j];
            if (v > bm) { bm = v; jm = j; }
          }
          // ties with the best are evaluated, so the lowest index wins them
          const bool want = (bm >= thr) && !(bm < best);
          if (!__any_sync(0xffffffffu, want)) break;
          if (want) xb[jm] = -INFINITY;
          float Zr[MAXM], Zi[MAXM];
#pragma unroll
          for (int m = 0; m < MAXM; ++m) { Zr[m] = 0.f; Zi[m] = 0.f; }
#pragma unroll 1
          for (int j = 0; j < EHALF; ++j) {
            if (!__any_sync(0xffffffffu, want && jm == j)) continue;
            float zr[MAXM], zi[MAXM];
#pragma unroll
            for (int m = 0; m < MAXM; ++m) {
              if (m < M) tmem_ld2(tbase + m * BN + 2 * (half * EHALF + j), zr[m], zi[m]);
              else { zr[m] = 0.f; zi[m] = 0.f; }
            }
            tmem_ld_wait();
            if (want && jm == j) {
#pragma unroll
              for (int m = 0; m < MAXM; ++m) { Zr[m] = zr[m]; Zi[m] = zi[m]; }
            }
          }
          if (want) {
            const int el = half * EHALF + jm;
            const int64_t e = e0 + el;
#pragma unroll
            for (int m = 0; m < MAXM; ++m) {
              Zr[m] *= zs;
              Zi[m] *= zs;
            }
            float C0, Cr[3], Ci[3];
            hh_tile<HH>(mrec, &T.qs[el * MAXD * REC], P, C0, Cr, Ci);
            int argo;
            const float ml = pair_ml(Zr, Zi, C0, Cr, Ci, thr, false, P, T.ph, argo);
            ++neval;
            const long long g = (i * P.n_ext + e) * (long long)P.n_phi + argo;
            if (ml > best || (ml == best && g < barg)) {
              best = ml;
              barg = g;
            }
          }
        }
        if (P.n_cand) {
          // here every pair taken is evaluated: both counters alike
          const int ne = __reduce_add_sync(0xffffffffu, neval);
          if (lane == 0 && ne > 0) {
            atomicAdd(&P.n_cand[0], (unsigned long long)ne);
            atomicAdd(&P.n_cand[1], (unsigned long long)ne);
          }
        }
        // the accumulators are no longer needed: release the buffer to the MMA warp
        tc_fence_before();
        __syncwarp();
        if (lane == 0) release_acc(b);
        // tile outputs of a screen: empty marginal partials and the tile's best ln L^ML
        warp_argmax(best, barg);
        if (lane == 0) {
          T.wml[ew] = best;
          T.warg[ew] = barg;
        }
        if (half == 0 && vi) P.row_part[(int64_t)et * P.n_int + i] = make_float2(-INFINITY, 0.f);
        if (etid < TE && e0 + etid < P.n_ext) P.col_part[(int64_t)it * P.n_ext + e0 + etid] = make_float2(-INFINITY, 0.f);
        named_bar_sync(1, EPT);
        if (etid == 0) {
          float bv = -1.f;
          long long bi = 0x7fffffffffffffffLL;
          for (int q = 0; q < NEPI; ++q)
            if (T.wml[q] > bv || (T.wml[q] == bv && T.warg[q] < bi)) { bv = T.wml[q]; bi = T.warg[q]; }
          P.tile_part[t] = make_float4(-INFINITY, 0.f, -INFINITY, 0.f);
          P.tile_ml[t] = bv;
          P.tile_arg[t] = bi;
          P.tile_npass[t] = 0;
          if (bv > 0.f && P.track_max) atomic_max_nonneg(P.ml_running, bv);
        }
        // the next tile's barrier (after its column records) orders these reads
        // of T.wml before any thread writes it again
        continue;
      } else {
#pragma unroll 1
      for (int j = 0; j < EHALF; ++j) {
        // SEP: samples of the first 16-sample half, then of the second (8 each)
        const int el = SEP ? (16 * (j >> 3) + 8 * half + (j & 7)) : (half * EHALF + j);
        const int64_t e = e0 + el;
        float Zr[MAXM], Zi[MAXM];
        if (SEP) {
          if (j == 8) {
            // the second half's accumulators
            if (!mbar_wait(&T.tfull[b], (use + 1) & 1, nullptr, abortp, wait_ns)) break;
            tc_fence_after();
          }
          // hi*hi in three interleaved sets, then the low-order set
          const uint32_t col = tbase + 2 * (8 * half + (j & 7));
          float Ar[4][MAXM], Ai[4][MAXM];
#pragma unroll
          for (int qs = 0; qs < 4; ++qs)
#pragma unroll
            for (int m = 0; m < MAXM; ++m) {
              if (m < M) tmem_ld2(col + qs * SEP_SET + m * SEP_N, Ar[qs][m], Ai[qs][m]);
              else { Ar[qs][m] = 0.f; Ai[qs][m] = 0.f; }
            }
          tmem_ld_wait();
#pragma unroll
          for (int m = 0; m < MAXM; ++m) {
            Zr[m] = ((Ar[0][m] + Ar[1][m]) + Ar[2][m]) + Ar[3][m];
            Zi[m] = ((Ai[0][m] + Ai[1][m]) + Ai[2][m]) + Ai[3][m];
          }
        } else {
#pragma unroll
          for (int m = 0; m < MAXM; ++m) {
            if (m < M) tmem_ld2(tbase + m * BN + 2 * el, Zr[m], Zi[m]);
            else { Zr[m] = 0.f; Zi[m] = 0.f; }
          }
          tmem_ld_wait();
        }
        if (j == EHALF - 1 || (SEP && j == 7)) {
          // this warp's accumulators are in registers: release the buffer to the MMA warp
          tc_fence_before();
          __syncwarp();
          if (lane == 0) release_acc(b);
        }
        float x = -INFINITY, x2 = -INFINITY;
        if (vi && e < P.n_ext) {
#pragma unroll
          for (int m = 0; m < MAXM; ++m) {
            Zr[m] *= zs;
            Zi[m] *= zs;
          }
          if (P.gemm_only) {
            float sx = 0.f;
#pragma unroll
            for (int m = 0; m < MAXM; ++m) sx += Zr[m] + Zi[m];
            x = sx;
            x2 = sx;
          } else if (P.screen_ml) {
            float C0, Cr[3], Ci[3];
            hh_tile<HH>(mrec, &T.qs[el * MAXD * REC], P, C0, Cr, Ci);
            int argo;
            const float ml = pair_ml(Zr, Zi, C0, Cr, Ci, thr, !store, P, T.ph, argo);
            if (ml > best) {
              best = ml;
              barg = (i * P.n_ext + e) * (long long)P.n_phi + argo;
            }
            if (store) {
              P.lnl_tile[i * P.n_ext + e] = -INFINITY;
              P.ml_tile[i * P.n_ext + e] = ml;
            }
          } else {
            float C0, Cr[3], Ci[3];
            hh_tile<HH>(mrec, &T.qs[el * MAXD * REC], P, C0, Cr, Ci);
            PairRes pr = pair_eval(Zr, Zi, C0, Cr, Ci, thr, !store, P, T.ph);
            const float lw = (float)(lwi + T.lwe[el]);
            x = pr.lsum + lw;
            x2 = pr.lsum2 + 2.f * lw;
            np += pr.npass;
            if (pr.ml > best) {
              best = pr.ml;
              barg = (i * P.n_ext + e) * (long long)P.n_phi + pr.argo;
            }
            if (store) {
              P.lnl_tile[i * P.n_ext + e] = pr.lsum - P.ln_nphi;
              P.ml_tile[i * P.n_ext + e] = pr.ml;
            }
          }
        }
        T.xs[row * XS_LD + el] = x;
        ra.add(x);
        rb.add(x2);
      }
      }
      if (half == 1) T.rowh[row] = make_float2(ra.m, ra.s);
      warp_merge_lse(rb);
      warp_argmax(best, barg);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) np += __shfl_xor_sync(0xffffffffu, np, o);
      {
        Lse w = ra;
        warp_merge_lse(w);
        if (lane == 0) {
          T.wm1[ew] = w.m; T.ws1[ew] = w.s; T.wm2[ew] = rb.m; T.ws2[ew] = rb.s;
          T.wml[ew] = best; T.warg[ew] = barg; T.wnp[ew] = np;
        }
      }
      named_bar_sync(1, EPT);
      if (half == 0 && vi && etv) {
        ra.merge(T.rowh[row].x, T.rowh[row].y);
        P.row_part[(int64_t)et * P.n_int + i] = make_float2(ra.m, ra.s);
      }
      {
        // column partials: 8 threads per extrinsic sample, 16 rows each
        const int cc = etid >> 3, qq = etid & 7;
        Lse a;
        a.init();
        for (int r = qq * 16; r < qq * 16 + 16; ++r) a.add(T.xs[r * XS_LD + cc]);
#pragma unroll
        for (int o = 1; o <= 4; o <<= 1) {
          float om = __shfl_xor_sync(0xffffffffu, a.m, o);
          float os = __shfl_xor_sync(0xffffffffu, a.s, o);
          a.merge(om, os);
        }
        if (qq == 0 && etv && e0 + cc < P.n_ext)
          P.col_part[(int64_t)it * P.n_ext + e0 + cc] = make_float2(a.m, a.s);
      }
      if (etid < 32 && etv) {
        // tile totals: lanes 0..NEPI-1 of the first epilogue warp hold the warps' values
        Lse a, bb;
        a.init();
        bb.init();
        float bv = -1.f;
        long long bi = 0x7fffffffffffffffLL;
        int n = 0;
        if (etid < NEPI) {
          a.merge(T.wm1[etid], T.ws1[etid]);
          bb.merge(T.wm2[etid], T.ws2[etid]);
          n = T.wnp[etid];
          bv = T.wml[etid];
          bi = T.warg[etid];
        }
        warp_merge_lse(a);
        warp_merge_lse(bb);
        warp_argmax(bv, bi);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
        if (etid == 0) {
          P.tile_part[t] = make_float4(a.m, a.s, bb.m, bb.s);
          P.tile_ml[t] = bv;
          P.tile_arg[t] = bi;
          P.tile_npass[t] = n;
          if (bv > 0.f && P.track_max) atomic_max_nonneg(P.ml_running, bv);
        }
      }
      // no trailing barrier: the next tile's barrier (after its column records)
      // orders these reads of the per-warp values before they are written again
      }  // TEV == 32
    }
  }
  tc_fence_before();
  __syncthreads();
  // a pair: neither CTA leaves while the other may still signal its barriers
  if constexpr (PAIR) cluster_sync_all();
  if (warp == 1) {
    if constexpr (PAIR) tmem_dealloc_pair(tmem, TMEM_COLS);
    else tmem_dealloc(tmem, TMEM_COLS);
  }
  // a wait that ran out leaves this CTA's tiles of every event unfinished
  if (threadIdx.x == 0 && T.abort_flag)
    for (int k = 0; k < Bt.n; ++k) atomicCAS(Bt.w[k].P.status, 0, DEV_E_TIMEOUT);
}

// Launches one instantiation chosen by the run-time flags (the kernel's
// parameter block is copied from *bt at launch).
template <int NB, bool SPLIT, bool SEP, int TEV>
cudaError_t launch_tc_variant(const TcLaunch &L, const TcBatch<NB> &bt, int grid, cudaStream_t st) {
  auto go = [&](auto kern) -> cudaError_t {
    const size_t smem = smem_bytes<SPLIT, TEV>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, NT, smem, st>>>(L.mapA, bt, L.C);
    return cudaGetLastError();
  };
  if (L.pol) {
    // polarisation-resolved banks run one event per launch, in 32-sample tiles
    if constexpr (NB == 1 && TEV == 32)
      return L.bf16 ? go(tc_fused_kernel<true, 2, SPLIT, NB, SEP, TEV>)
                    : go(tc_fused_kernel<false, 2, SPLIT, NB, SEP, TEV>);
    else
      return cudaErrorInvalidValue;
  }
  if constexpr (NB == 1 && TEV == 64 && !SPLIT) {
    if (L.pair) {
      // clusters of two CTAs (grid even)
      auto go2 = [&](auto kern) -> cudaError_t {
        const size_t smem = smem_bytes<false, 64, true>();
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)grid, 1, 1);
        cfg.blockDim = dim3(NT, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        // no more pairs than can be resident at once (a persistent grid: a pair that
        // waited for another to finish would add its whole share to the tail)
        static int max_pairs = 0;
        if (max_pairs == 0) {
          int mc = 0;
          if (cudaOccupancyMaxActiveClusters(&mc, kern, &cfg) != cudaSuccess || mc < 1) {
            cudaGetLastError();
            mc = grid / 2;
          }
          max_pairs = mc;
        }
        if (grid / 2 > max_pairs) cfg.gridDim.x = 2u * (unsigned)max_pairs;
        e = cudaLaunchKernelEx(&cfg, kern, L.mapA, bt, L.C);
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
      };
      if (grid % 2 != 0) return cudaErrorInvalidValue;
      if (L.bf16) return L.consec ? go2(tc_fused_kernel<true, 1, false, 1, false, 64, true>)
                                  : go2(tc_fused_kernel<true, 0, false, 1, false, 64, true>);
      return L.consec ? go2(tc_fused_kernel<false, 1, false, 1, false, 64, true>)
                      : go2(tc_fused_kernel<false, 0, false, 1, false, 64, true>);
    }
  }
  if (L.bf16) return L.consec ? go(tc_fused_kernel<true, 1, SPLIT, NB, SEP, TEV>)
                              : go(tc_fused_kernel<true, 0, SPLIT, NB, SEP, TEV>);
  return L.consec ? go(tc_fused_kernel<false, 1, SPLIT, NB, SEP, TEV>)
                  : go(tc_fused_kernel<false, 0, SPLIT, NB, SEP, TEV>);
}

template <int NB>
cudaError_t launch_tc_any(const TcLaunch &L, const TcBatch<NB> &bt, int grid, cudaStream_t st) {
  if (L.tev == 64) {
    // 64-sample work tiles: single pass, grid order only (no device list)
    if (L.split || L.pol || bt.glist) return cudaErrorInvalidValue;
    return launch_tc_variant<NB, false, false, 64>(L, bt, grid, st);
  }
  if (!L.split) return launch_tc_variant<NB, false, false, 32>(L, bt, grid, st);
  return L.sep ? launch_tc_variant<NB, true, true, 32>(L, bt, grid, st)
               : launch_tc_variant<NB, true, false, 32>(L, bt, grid, st);
}

}  // namespace dotpe
