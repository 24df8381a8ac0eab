// Incoherent single-detector pre-selection (Sec. IV.D, App. B) on the
// 5th-generation tensor cores.
//
// For bank row i, detector k, arrival time t_{kt} and orbital phase phi_o:
//   Z_{ikmt}        = sum_b h_{im}(f_b) c_{kb} e^{-2 pi i f_b t_{kt}}     (Eq. dh_itop, per mode)
//   <d|h>_{iktop}   = Re sum_m e^{i m phi_o} K_{imp} Z_{ikmt}
//   <h|h>_{ikopp'}  = Re sum_{m,m'} K_{imp} K^*_{im'p'} e^{i (m - m') phi_o} <h_m|h_m'>_k
//   ln L^ML_{ikot}  = dh^T [hh]^+ dh / 2                                   (Eqs. x_ML, single_det_ML)
// with K_{imp} the row's polarisation factors (h_{imp} = K_{imp} h_{im}).
// The kernel keeps, per (i, k), the maximum over (o, t) and its (o, t); the
// sum over detectors and the selection window of Sec. IV.D follow in two
// small kernels.  [hh]^+ is the inverse when det > rank_tol hh_{++} hh_{xx},
// else the rank-one pseudo-inverse hh / (hh_{++} + hh_{xx})^2.
//
// Z is a real-ified complex GEMM, one MMA per k-step covering every mode:
//   A (M = 128 lanes) = the time-grid operand G_k[b, t] = c_{kb} e^{-2 pi i f_b t_{kt}},
//       rows [(k, t) re-row; (k, t) im-row] x [re | im]: 64 (k, t) columns per tile;
//   B (N = 64 M) = 64 bank rows of each mode, the bank's own operand planes
//       (one TMA box per mode, stacked in shared memory mode after mode).
// With relative binning (App. A) the data weights, hence G, differ per mode
// (PERMODE): a stage then holds one mode's A and B and each MMA is N = 64
// into that mode's TMEM columns.
// TMEM lane 2c + part holds Re (part 0) or Im (part 1) of column c's Z; TMEM
// column 64 m + j holds bank row j of mode m.  The small G operand stays in
// L2; the bank streams from HBM, each row block once for all its column tiles
// (they are neighbours in the schedule).  Persistent and warp-specialised:
//   warp 0       TMA producer
//   warp 1       TMEM allocator and tcgen05.mma issuer (lane 0)
//   warps 2..17  epilogue: four warps per TMEM lane quadrant, 16 bank rows each
// Two TMEM buffers of 256 columns.  Each detector's time grid is padded to a
// multiple of 64 columns, so a tile lies in one detector.
//
// Epilogue.  Per tile the 512 epilogue threads first tabulate [hh]^+ / 2 of the
// tile's 64 rows on every phase in shared memory: for a mode bank 192 threads
// (row, polarisation pair) form the row's phase-independent coefficients of
// <h|h>_{pp'}(phi) once, then every thread evaluates one (row, 4 phases).
// Then each lane takes its column (one arrival time; its TMEM lane holds the
// Re or the Im part) and the warp's 16 rows: it reads the mode components from
// TMEM and, for a mode bank, swaps with the partner lane the parts of two rows
// so that it holds the whole Z of every other row (the partner the rest), forms
// Y_{mp} = K_{mp} Z_m and evaluates all phases of its rows.  (A polarisation-
// resolved bank keeps four lanes per column, each with a quarter of the
// phases.)  With n_phi a multiple of 4 one rotation serves several phases: a
// mode bank (distinct m in 1..4, one per class m mod 4) takes them in
// quadruples (phi + k pi / 2, k = 0..3) from e^{i m (phi + pi / 2)} =
// i^m e^{i m phi}; a polarisation-resolved bank in pairs (phi, phi + pi), with
// the modes ordered even m first, from e^{i m (phi + pi)} = +-e^{i m phi}.
// The row's best (ln L^ML, o) over
// the warp's 16 times is a warp reduction, merged across tiles with a 64-bit
// atomic maximum.  The phase index rides in the low 6 mantissa bits of
// ln L^ML (a change of at most 2^-17 of the value), so the inner maximum is one
// FMNMX.
#pragma once
#include "common.cuh"
#include "kernels.h"

namespace dotpe {

namespace {
constexpr int QTR = PS_TR;          // bank rows per tile
constexpr int QTC = PS_TC;          // (detector, time) columns per tile
constexpr int QBM = 2 * QTC;        // A rows (re, im) = MMA M
static_assert(QBM == 128, "one TMEM lane per A row");
constexpr int QBK = 64;
constexpr int QNEPI = 16;           // epilogue warps
constexpr int QNT = (2 + QNEPI) * 32;
constexpr int QEPT = QNEPI * 32;
constexpr int QJW = QTR / 4;        // bank rows per epilogue warp
constexpr int QJC = 8;              // bank rows per TMEM load
static_assert(QEPT == QTR * 8 && PS_MAXPHI == 32, "table pass: one thread per (row, 4 phases)");
constexpr uint32_t QA_BYTES = QBM * QBK * 2;             // 16 KB per plane
constexpr uint32_t QB_MODE = QTR * QBK * 2;              // 8 KB per mode and plane
constexpr uint32_t QB_BYTES = MAXM * QB_MODE;            // 32 KB per plane
// Stage = one k-block of A and of all modes' B (shared time-grid operand), or,
// PERMODE (a time-grid operand per mode: relative binning), one k-block of one
// mode's A and B.  Both fill 192 KB.
template <bool SPLIT, bool PERMODE> struct QPipe {
  static constexpr int NPL = SPLIT ? 2 : 1;
  static constexpr uint32_t BSZ = PERMODE ? QB_MODE : QB_BYTES;  // B bytes per plane and stage
  static constexpr int ST = PERMODE ? (SPLIT ? 4 : 8) : (SPLIT ? 2 : 4);
  static constexpr uint32_t STAGE = NPL * (QA_BYTES + BSZ);
};
constexpr uint32_t Q_TMEM_COLS = 512, Q_BUF_COLS = MAXM * QTR;
static_assert(2 * Q_BUF_COLS <= Q_TMEM_COLS, "TMEM budget");

struct QTail {
  float4 hs[QTR * PS_MAXPHI];       // [row][o]: (a, 2b, c, -), ln L^ML = a dp^2 + 2b dp dx + c dx^2
  float4 phm[PS_MAXPHI * 2];        // (cos, sin)(m_s phi_o) of the four mode slots: [o][(c0, s0, c1, s1), (c2, s2, c3, s3)]
  float2 phd[PS_MAXPHI * 3];        // (cos, sin)(delta phi_o), delta = 1..3
  uint64_t full[8], empty[8], tfull[2], tempty[2], drain;
  uint32_t tmem_slot;
  int abort_flag;
};
template <bool SPLIT, bool PERMODE>
constexpr size_t q_smem_bytes() {
  return 1024 + (size_t)QPipe<SPLIT, PERMODE>::ST * QPipe<SPLIT, PERMODE>::STAGE + sizeof(QTail);
}
static_assert(q_smem_bytes<true, false>() <= 232448 && q_smem_bytes<false, false>() <= 232448 &&
                  q_smem_bytes<true, true>() <= 232448 && q_smem_bytes<false, true>() <= 232448,
              "shared memory budget");
static_assert(QPipe<false, true>::ST <= 8, "stage barriers");

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = __uint_as_float(r[k]);
}

// ln L^ML with the phase code in the low 6 mantissa bits (larger code = lower
// phase, so ties keep the lowest phase).
__device__ __forceinline__ float tag(float q, int code) {
  return __int_as_float((__float_as_int(q) & ~63) | code);
}

// Re(Y_s e^{i m_s phi}) summed over the even-mode slots [0, NE) and the odd
// ones [NE, MAXM), for one polarisation: E +- O is <d|h> at phi and phi + pi.
template <int NE>
__device__ __forceinline__ void even_odd(const float4 &e01, const float4 &e23, const float *yr, const float *yi,
                                         float &E, float &O) {
  const float r0 = e01.x * yr[0] - e01.y * yi[0];
  const float r1 = e01.z * yr[1] - e01.w * yi[1];
  const float r2 = e23.x * yr[2] - e23.y * yi[2];
  const float r3 = e23.z * yr[3] - e23.w * yi[3];
  if (NE == 0) { E = 0.f; O = (r0 + r1) + (r2 + r3); }
  else if (NE == 1) { E = r0; O = r1 + (r2 + r3); }
  else if (NE == 2) { E = r0 + r1; O = r2 + r3; }
  else if (NE == 3) { E = (r0 + r1) + r2; O = r3; }
  else { E = (r0 + r1) + (r2 + r3); O = 0.f; }
}

// Re sum_s Y_s e^{i m_s (phi + k pi / 2)}, k = 0..3, for one polarisation, the
// slots holding the classes m mod 4 = 0, 2, 1, 3 (i^m = 1, -1, i, -i):
// with R_c = Re(Y e^{i m phi}) and P_c = Y e^{i m phi} of class c,
//   d0 = (R_0 + R_2) + (Re P_1 + Re P_3),   d1 = (R_0 - R_2) + (Im P_3 - Im P_1),
//   d2 = (R_0 + R_2) - (Re P_1 + Re P_3),   d3 = (R_0 - R_2) - (Im P_3 - Im P_1).
__device__ __forceinline__ void quarter_turns(const float4 &e01, const float4 &e23, const float *yr, const float *yi,
                                              float (&d)[4]) {
  const float r0 = e01.x * yr[0] - e01.y * yi[0];
  const float r2 = e01.z * yr[1] - e01.w * yi[1];
  const float p1r = e23.x * yr[2] - e23.y * yi[2], p1i = e23.x * yi[2] + e23.y * yr[2];
  const float p3r = e23.z * yr[3] - e23.w * yi[3], p3i = e23.z * yi[3] + e23.w * yr[3];
  const float a = r0 + r2, b = r0 - r2, c = p1r + p3r, e = p3i - p1i;
  d[0] = a + c; d[1] = b + e; d[2] = a - c; d[3] = b - e;
}
}  // namespace

// One row of one column: best tagged ln L^ML over the thread's phases.
// PH 2 (quarter turns; n_phi % 4 == 0, slots by class m mod 4): base phases
// b = part, part + STEP, ... < n_phi / 4 and b + k n_phi / 4; PH 1 (pairs;
// n_phi % 4 == 0): base phases b < n_phi / 2 and their partners b + n_phi / 2;
// PH 0: phases o = part, part + STEP, ...  (STEP lanes share one (row, time):
// 1 for a mode bank, 4 for a polarisation-resolved bank; PH 2 takes every
// phase.)  With PH 2 and n_phi / 4 even the base phases go in pairs, in the
// order (c + sw, c + 1 - sw): the lanes of a warp that read two rows at once
// (512 bytes apart in the table) with sw = 0 and 1 then read different
// phases, in different shared-memory banks.
template <int NE, int PH, int STEP>
__device__ __forceinline__ float row_best(const float (&yr)[MAXM][2], const float (&yi)[MAXM][2],
                                          const float4 *__restrict__ hs_row, const QTail &T, int n_phi, int part,
                                          int sw = 0) {
  float best = -1.f;
  float yrp[MAXM], yip[MAXM], yrx[MAXM], yix[MAXM];
#pragma unroll
  for (int s = 0; s < MAXM; ++s) { yrp[s] = yr[s][0]; yip[s] = yi[s][0]; yrx[s] = yr[s][1]; yix[s] = yi[s][1]; }
  if (PH == 2) {
    const int qn = n_phi >> 2;
    // one base phase b: <d|h> of both polarisations at b + k qn, k = 0..3, from one
    // rotation; ph = the phase table at b, hq = the row's table entry at b, code0 = 63 - b
    auto quad_step = [&](const float4 *ph, const float4 *hq, int code0) {
      const float4 e01 = ph[0], e23 = ph[1];
      float dp[4], dx[4];
      quarter_turns(e01, e23, yrp, yip, dp);
      quarter_turns(e01, e23, yrx, yix, dx);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float4 h = hq[k * qn];
        const float q = fmaf(dp[k], fmaf(h.y, dx[k], h.x * dp[k]), h.z * dx[k] * dx[k]);
        best = fmaxf(best, tag(q, code0 - k * qn));
      }
    };
    if (qn & 1) {
#pragma unroll 2
      for (int b = 0; b < qn; ++b) quad_step(T.phm + 2 * b, hs_row + b, 63 - b);
    } else {
      // base phases in pairs (c + sw, c + 1 - sw): the per-lane offset sw is folded
      // into the pointers, so the swizzle costs nothing inside the loop
      const float4 *pA = T.phm + 2 * sw, *pB = T.phm + 2 * (1 - sw);
      const float4 *hA = hs_row + sw, *hB = hs_row + (1 - sw);
#pragma unroll 1
      for (int c = 0; c < qn; c += 2) {
        quad_step(pA + 2 * c, hA + c, 63 - sw - c);
        quad_step(pB + 2 * c, hB + c, 62 + sw - c);
      }
    }
  } else if (PH == 1) {
    const int half = n_phi >> 1;
#pragma unroll 4
    for (int b = part; b < half; b += STEP) {
      const float4 e01 = T.phm[b * 2], e23 = T.phm[b * 2 + 1];
      float Ep, Op, Ex, Ox;
      even_odd<NE>(e01, e23, yrp, yip, Ep, Op);
      even_odd<NE>(e01, e23, yrx, yix, Ex, Ox);
      const float4 h0 = hs_row[b], h1 = hs_row[b + half];
      const float dp0 = Ep + Op, dx0 = Ex + Ox, dp1 = Ep - Op, dx1 = Ex - Ox;
      const float q0 = fmaf(dp0, fmaf(h0.y, dx0, h0.x * dp0), h0.z * dx0 * dx0);
      const float q1 = fmaf(dp1, fmaf(h1.y, dx1, h1.x * dp1), h1.z * dx1 * dx1);
      best = fmaxf(best, fmaxf(tag(q0, 63 - b), tag(q1, 63 - (b + half))));
    }
  } else {
#pragma unroll 2
    for (int o = part; o < n_phi; o += STEP) {
      const float4 e01 = T.phm[o * 2], e23 = T.phm[o * 2 + 1];
      float Ep, Op, Ex, Ox;
      even_odd<NE>(e01, e23, yrp, yip, Ep, Op);
      even_odd<NE>(e01, e23, yrx, yix, Ex, Ox);
      const float4 h = hs_row[o];
      const float dp = Ep + Op, dx = Ex + Ox;
      const float q = fmaf(dp, fmaf(h.y, dx, h.x * dp), h.z * dx * dx);
      best = fmaxf(best, tag(q, 63 - o));
    }
  }
  return best;
}

// The warp's 16 rows of one tile of a mode bank for the lane's column t: mode
// components from TMEM (the buffer is released after the last read); of each
// two rows the Re lane (part 0) takes the first and the Im lane the second,
// the two swapping the parts each lacks, so each lane holds the whole Z of its
// rows; Y = K Z (the accumulator scale is in the [hh]^+ table), the best tagged
// ln L^ML over every phase, the maximum over the warp's 16 times (the lanes of
// one part), one atomic per row.
template <int PH>
__device__ __forceinline__ void tile_rows_modes(const PreselParams &P, const QTail &T, uint32_t tbase, int rb,
                                                int j_first, int k, int t, int part, int lane, uint64_t *tempty) {
  const bool tv = t < P.n_t;
  const int sw = ((P.n_phi >> 2) & 1) ? 0 : part;  // phase order of the odd rows (see row_best)
#pragma unroll 1
  for (int jc = 0; jc < QJW / QJC; ++jc) {
    const int j0 = j_first + jc * QJC;
    float z[MAXM][QJC];
#pragma unroll
    for (int s = 0; s < MAXM; ++s) {
      if ((P.slot_mask >> s) & 1u) tmem_ld8(tbase + P.slot[s] * QTR + j0, z[s]);
      else {
#pragma unroll
        for (int q = 0; q < QJC; ++q) z[s][q] = 0.f;
      }
    }
    tmem_ld_wait();
    if (jc == QJW / QJC - 1) {
      // this warp's last read of the buffer: release it to the MMA warp
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty);
    }
#pragma unroll
    for (int r = 0; r < QJC / 2; ++r) {
      const int j = j0 + 2 * r + part;  // this lane's row
      const int64_t i = (int64_t)rb * QTR + j;
      const bool rv = i < P.n_rows;
      float zr[MAXM], zi[MAXM];
#pragma unroll
      for (int s = 0; s < MAXM; ++s) {
        // the Re lane holds Re of rows 2r, 2r + 1, the Im lane their Im: each
        // sends the part of the partner's row
        const float send = part ? z[s][2 * r] : z[s][2 * r + 1];
        const float recv = __shfl_xor_sync(0xffffffffu, send, 1);
        zr[s] = part ? recv : z[s][2 * r];
        zi[s] = part ? z[s][2 * r + 1] : recv;
      }
      // the row's polarisation factors from the fourth words of its table
      // entries 4 s + c + (j & 1) (zero for empty slots)
      const float *kw = reinterpret_cast<const float *>(&T.hs[j * PS_MAXPHI + part]) + 3;
      float yr[MAXM][2], yi[MAXM][2];
#pragma unroll
      for (int s = 0; s < MAXM; ++s) {
        const float4 kv = make_float4(kw[16 * s], kw[16 * s + 4], kw[16 * s + 8], kw[16 * s + 12]);
        yr[s][0] = kv.x * zr[s] - kv.y * zi[s];
        yi[s][0] = kv.x * zi[s] + kv.y * zr[s];
        yr[s][1] = kv.z * zr[s] - kv.w * zi[s];
        yi[s][1] = kv.z * zi[s] + kv.w * zr[s];
      }
      const float best = row_best<0, PH, 1>(yr, yi, &T.hs[j * PS_MAXPHI], T, P.n_phi, 0, sw);
      // the maximum over the warp's 16 times of this lane's row (lanes of the
      // same part): tagged values are distinct between the phases of one time, so
      // the lowest lane holding the maximum has the lowest time
      const bool ok = tv && rv;
      float m = ok ? best : -1.f;
#pragma unroll
      for (int sh = 16; sh > 1; sh >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, sh));
      const unsigned hit = __ballot_sync(0xffffffffu, ok && best == m) & (part ? 0xAAAAAAAAu : 0x55555555u);
      if (lane < 2 && m >= -0.5f && hit) {
        const int t_hit = t + ((__ffs(hit) - 1) >> 1);  // lane 0's (= lane 1's) time + the lane offset's time
        const uint32_t o = 63u - (uint32_t)(__float_as_int(m) & 63);
        const unsigned long long key = ((unsigned long long)__float_as_uint(fmaxf(m, 0.f)) << 32) |
                                       (unsigned long long)(0xffffffffu - (uint32_t)(t_hit * P.n_phi + (int)o));
        atomicMax(P.keys + i * P.n_det + k, key);
      }
    }
  }
}

// The warp's 16 rows of one tile of a polarisation-resolved bank: lanes
// 4c + 2p + part hold (Re, Im) of the (mode, polarisation p) component of
// column c; the four lanes of a column exchange their parts, take
// Y_{mp} = Z_{mp} (no factors) and a quarter of the phases each, then the warp
// maximum over its 8 times and one atomic per row.
template <int NE, int PH>
__device__ __forceinline__ void tile_rows_pol(const PreselParams &P, const QTail &T, uint32_t tbase, int rb,
                                              int j_first, int k, int t, int part, int lane, uint64_t *tempty) {
  const bool tv = t < P.n_t;
#pragma unroll 1
  for (int jc = 0; jc < QJW / QJC; ++jc) {
    const int j0 = j_first + jc * QJC;
    float z[MAXM][QJC];
#pragma unroll
    for (int s = 0; s < MAXM; ++s) {
      if ((P.slot_mask >> s) & 1u) tmem_ld8(tbase + P.slot[s] * QTR + j0, z[s]);
      else {
#pragma unroll
        for (int q = 0; q < QJC; ++q) z[s][q] = 0.f;
      }
    }
    tmem_ld_wait();
    if (jc == QJW / QJC - 1) {
      // this warp's last read of the buffer: release it to the MMA warp
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty);
    }
#pragma unroll
    for (int jj = 0; jj < QJC; ++jj) {
      const int j = j0 + jj;
      const int64_t i = (int64_t)rb * QTR + j;
      float yr[MAXM][2], yi[MAXM][2];
      const int pp = (lane >> 1) & 1;
#pragma unroll
      for (int s = 0; s < MAXM; ++s) {
        const float own = z[s][jj];
        const float x1 = __shfl_xor_sync(0xffffffffu, own, 1);  // (p, other part)
        const float x2 = __shfl_xor_sync(0xffffffffu, own, 2);  // (other p, this part)
        const float x3 = __shfl_xor_sync(0xffffffffu, own, 3);  // (other p, other part)
        const float r_own = part ? x1 : own, i_own = part ? own : x1;
        const float r_oth = part ? x3 : x2, i_oth = part ? x2 : x3;
        yr[s][0] = pp ? r_oth : r_own; yi[s][0] = pp ? i_oth : i_own;
        yr[s][1] = pp ? r_own : r_oth; yi[s][1] = pp ? i_own : i_oth;
      }
      if (i >= P.n_rows) continue;  // warp-uniform
      const float best = row_best<NE, PH, 4>(yr, yi, &T.hs[j * PS_MAXPHI], T, P.n_phi, lane & 3);
      // the warp's maximum over its 8 times: tagged values are distinct between
      // the lanes of one time, so the lowest lane holding the maximum has the
      // lowest time
      float m = tv ? best : -1.f;
#pragma unroll
      for (int sh = 16; sh > 0; sh >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, sh));
      const unsigned hit = __ballot_sync(0xffffffffu, tv && best == m);
      if (lane == 0 && m >= -0.5f && hit) {
        const int t_hit = t + ((__ffs(hit) - 1) >> 2);  // lane 0's time + the lane offset's time
        const uint32_t o = 63u - (uint32_t)(__float_as_int(m) & 63);
        const unsigned long long key = ((unsigned long long)__float_as_uint(fmaxf(m, 0.f)) << 32) |
                                       (unsigned long long)(0xffffffffu - (uint32_t)(t_hit * P.n_phi + (int)o));
        atomicMax(P.keys + i * P.n_det + k, key);
      }
    }
  }
}

// VAR: 0 shared time-grid operand, 1 one per mode (relative binning), 2
// polarisation-resolved bank (A rows 4c + 2p + part: 32 columns per tile).
template <bool BF16, bool SPLIT, int VAR>
__global__ void __launch_bounds__(QNT, 1)
    presel_kernel(const __grid_constant__ CUtensorMap mapG, const __grid_constant__ CUtensorMap mapBank,
                  const __grid_constant__ PreselParams P) {
  constexpr bool PERMODE = (VAR == 1), POL = (VAR == 2);
  constexpr int QCOLS = POL ? QTC / 2 : QTC;  // (detector, time) columns per tile
  using Pipe = QPipe<SPLIT, PERMODE>;
  constexpr int ST = Pipe::ST, NPL = Pipe::NPL;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // stage s, plane p: A (G, 16 KB) then B (bank: all modes, 4 x 8 KB, or PERMODE one mode, 8 KB)
  QTail &T = *reinterpret_cast<QTail *>(base + (size_t)ST * Pipe::STAGE);
  auto sA = [&](int s, int p) { return base + (size_t)(s * NPL + p) * (QA_BYTES + Pipe::BSZ); };
  auto sB = [&](int s, int p) { return sA(s, p) + QA_BYTES; };
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int M = P.n_modes;
  const int n_work = P.n_itile * P.n_ctile;
  const int nkb = P.kb;
  const int nsub = PERMODE ? M : 1;  // stages per k-block
  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(&T.full[s], 1);
      mbar_init(&T.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&T.tfull[b], 1);
      mbar_init(&T.tempty[b], QNEPI);
    }
    mbar_init(&T.drain, 1);
    T.abort_flag = 0;
    mbar_fence_init();
  }
  // phase tables, mode slots in the order of P.slot (angles reduced in integers first)
  for (int q = threadIdx.x; q < PS_MAXPHI * 4; q += QNT) {
    const int o = q >> 2, s = q & 3;
    float c = 1.f, sn = 0.f, c2 = 1.f, s2 = 0.f;
    if (o < P.n_phi) {
      const int mm = ((P.slot_mask >> s) & 1u) ? P.mode_m[P.slot[s]] : 0;
      sincospif(2.0f * (float)((mm * o) % P.n_phi) / (float)P.n_phi, &sn, &c);
      sincospif(2.0f * (float)((s * o) % P.n_phi) / (float)P.n_phi, &s2, &c2);
    }
    float *pm = reinterpret_cast<float *>(&T.phm[o * 2]);
    pm[2 * s] = c;
    pm[2 * s + 1] = sn;
    if (s > 0) T.phd[o * 3 + s - 1] = make_float2(c2, s2);
  }
  if (warp == 0 && lane == 0) {
    tma_prefetch_desc(&mapG);
    tma_prefetch_desc(&mapBank);
  }
  if (warp == 1) tmem_alloc(&T.tmem_slot, Q_TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = T.tmem_slot;
  volatile int *abortp = &T.abort_flag;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      const uint32_t stage_bytes = PERMODE ? NPL * (QA_BYTES + QB_MODE) : NPL * (QA_BYTES + M * QB_MODE);
      uint32_t q = 0;
      bool ok = true;
      for (int w = blockIdx.x; w < n_work && ok; w += gridDim.x) {
        const int rb = w / P.n_ctile, ct = w - rb * P.n_ctile;
        for (int kb = 0; kb < nkb && ok; ++kb)
          for (int sub = 0; sub < nsub; ++sub, ++q) {
            const int s = q % ST;
            const uint32_t n = q / ST;
            if (n > 0 && !(ok = mbar_wait(&T.empty[s], (n - 1) & 1, nullptr, abortp, P.wait_ns))) break;
            mbar_expect_tx(&T.full[s], stage_bytes);
#pragma unroll
            for (int pl = 0; pl < NPL; ++pl) {
              tma_load_3d(sA(s, pl), &mapG, &T.full[s], 0, pl * P.b_plane_rows + sub * P.b_mode_rows + ct * QBM, kb);
              const int m0 = PERMODE ? sub : 0, m1 = PERMODE ? sub + 1 : M;
              for (int m = m0; m < m1; ++m)
                tma_load_3d(sB(s, pl) + (m - m0) * QB_MODE, &mapBank, &T.full[s], 0,
                            pl * P.a_plane_rows + m * P.a_mode_rows + P.a_row0 + rb * QTR, kb);
            }
          }
      }
      if (!ok) {
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
    const uint32_t idesc = idesc_f16(128, PERMODE ? QTR : QTR * M, BF16);
    const bool issuer = (lane == 0);
    uint32_t q = 0, u = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < n_work && ok; w += gridDim.x) {
      const int b = u & 1;
      const uint32_t use = u >> 1;
      ++u;
      if (use > 0) ok = __all_sync(0xffffffffu, mbar_wait(&T.tempty[b], (use - 1) & 1, nullptr, abortp, P.wait_ns));
      if (!ok) break;
      tc_fence_after();
      for (int kb = 0; kb < nkb && ok; ++kb)
        for (int sub = 0; sub < nsub; ++sub, ++q) {
          const int s = q % ST;
          const uint32_t n = q / ST;
          ok = __all_sync(0xffffffffu, mbar_wait(&T.full[s], n & 1, nullptr, abortp, P.wait_ns));
          if (!ok) break;
          tc_fence_after();
          if (issuer) {
            const uint32_t dcol = tmem + b * Q_BUF_COLS + (PERMODE ? sub * QTR : 0);
            const uint64_t ah = sdesc_k128(sA(s, 0)), bh = sdesc_k128(sB(s, 0));
            const uint64_t al = sdesc_k128(sA(s, NPL - 1)), bl = sdesc_k128(sB(s, NPL - 1));
#pragma unroll
            for (int k = 0; k < QBK / 16; ++k) {
              tc_mma(dcol, ah + 2 * k, bh + 2 * k, idesc, (kb | k) ? 1u : 0u);
              if (SPLIT) {
                tc_mma(dcol, ah + 2 * k, bl + 2 * k, idesc, 1u);  // hi * lo
                tc_mma(dcol, al + 2 * k, bh + 2 * k, idesc, 1u);  // lo * hi
              }
            }
            tc_commit(&T.empty[s]);
          }
          __syncwarp();
        }
      if (ok && issuer) tc_commit(&T.tfull[b]);
      __syncwarp();
    }
    if (issuer) tc_commit(&T.drain);
    __syncwarp();
    volatile int no_abort = 0;
    mbar_wait(&T.drain, 0, nullptr, &no_abort, 500000000ull);
  } else {
    // ---------------- epilogue ----------------
    const int ew = warp - 2;               // 0..15
    const int quad = warp & 3;             // TMEM lane quadrant
    const int sub = ew >> 2;               // which 16 rows of the tile
    const int etid = threadIdx.x - 64;
    const int L = quad * 32 + lane;        // TMEM lane = A row
    const int part = L & 1;                // 0: Re row, 1: Im row
    const float zs = P.z_scale / (P.g_scale ? *P.g_scale : 1.f);
    const float zs2 = zs * zs;
    const bool pair = (P.n_phi & 3) == 0;
    uint32_t u = 0;
    for (int w = blockIdx.x; w < n_work; w += gridDim.x) {
      const int rb = w / P.n_ctile, ct = w - rb * P.n_ctile;
      const int b = u & 1;
      const uint32_t use = u >> 1;
      ++u;
      const int c0 = ct * QCOLS;
      const int k = c0 / P.n_tpad;
      // ---- [hh]^+ / 2 of the tile's rows on every phase (thread = row, 4 phases)
      named_bar_sync(1, QEPT);  // the previous tile's readers are done with T.hs
      {
        const int j = etid >> 3, o0 = (etid & 7) * 4;
        const int64_t i = (int64_t)rb * QTR + j;
        if (POL && i < P.n_rows && o0 < P.n_phi) {
          // the row's records (grouped by delta = m - m'): hh_{++} = X0 + 2 Re sum X_d e^{i d phi},
          // hh_{xx} = W0 + 2 Re sum W_d e^{i d phi}, hh_{+x} = Y0 / 2 + Re sum Y_d e^{i d phi}
          const float *rec = P.mx + (i * P.n_det + k) * REC_P;
          float rv[REC_POL];
#pragma unroll
          for (int q = 0; q < REC_POL; ++q) rv[q] = __ldg(rec + q);
#pragma unroll
          for (int oo = 0; oo < 4; ++oo) {
            const int o = o0 + oo;
            float A = rv[0], Bx = 0.5f * rv[1], C = rv[2];
#pragma unroll
            for (int dl = 0; dl < 3; ++dl) {
              const float2 e = T.phd[o * 3 + dl];
              A += 2.f * (rv[3 + 6 * dl] * e.x - rv[4 + 6 * dl] * e.y);
              Bx += rv[5 + 6 * dl] * e.x - rv[6 + 6 * dl] * e.y;
              C += 2.f * (rv[7 + 6 * dl] * e.x - rv[8 + 6 * dl] * e.y);
            }
            const float det = A * C - Bx * Bx;
            float a = 0.f, bb = 0.f, c = 0.f;
            if (det > P.rank_tol * A * C) {
              const float inv = 0.5f / det;
              a = C * inv; bb = -Bx * inv; c = A * inv;
            } else if (A > 0.f || C > 0.f) {
              const float sm = A + C;
              const float inv = 0.5f / (sm * sm);
              a = A * inv; bb = Bx * inv; c = C * inv;
            }
            T.hs[j * PS_MAXPHI + o] = make_float4(a * zs2, 2.f * bb * zs2, c * zs2, 0.f);
          }
        }
        if constexpr (!POL) {
          // <h|h>_{pp'}(phi) = Dc_r + sum_delta Re(Q_r[delta] e^{i delta phi}), r = (++, +x, xx):
          // (a) one thread per (row, r) forms the row's coefficients (Dc_r, Re Q_r, Im Q_r)
          // into the row's own part of T.hs (rows of one warp 8 words apart, so that
          // the reads of (b) meet distinct banks)
          if (etid < QTR * 3) {
            const int ja = etid / 3, r = etid - 3 * ja;
            const int64_t ia = (int64_t)rb * QTR + ja;
            if (ia < P.n_rows) {
              // K_{mp} and K_{mp'} of the thread's polarisation pair (p, p')
              const bool p1 = r == 2, pp1 = r != 0;
              float Kpr[MAXM], Kpi[MAXM], Kqr[MAXM], Kqi[MAXM], rec[REC];
#pragma unroll
              for (int m = 0; m < MAXM; ++m) {
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (m < M) v = __ldg(reinterpret_cast<const float4 *>(P.pol + (ia * M + m) * 2));
                Kpr[m] = p1 ? v.z : v.x; Kpi[m] = p1 ? v.w : v.y;
                Kqr[m] = pp1 ? v.z : v.x; Kqi[m] = pp1 ? v.w : v.y;
              }
              const float4 *src = reinterpret_cast<const float4 *>(P.mx + (ia * P.n_det + k) * REC);
#pragma unroll
              for (int q = 0; q < REC / 4; ++q) {
                const float4 v = __ldg(src + q);
                rec[4 * q] = v.x; rec[4 * q + 1] = v.y; rec[4 * q + 2] = v.z; rec[4 * q + 3] = v.w;
              }
              float Dc = 0.f, Qr[3] = {0.f, 0.f, 0.f}, Qi[3] = {0.f, 0.f, 0.f};
#pragma unroll
              for (int m = 0; m < MAXM; ++m) Dc += rec[m] * (Kpr[m] * Kqr[m] + Kpi[m] * Kqi[m]);
              int pr = 0;
#pragma unroll
              for (int a = 1; a < MAXM; ++a)
#pragma unroll
                for (int c = 0; c < a; ++c, ++pr) {
                  if (a >= M) continue;
                  // X = K_ap K_cp'^* + K_ap' K_cp^*, times <h_a|h_c>
                  const float xr = Kpr[a] * Kqr[c] + Kpi[a] * Kqi[c] + Kqr[a] * Kpr[c] + Kqi[a] * Kpi[c];
                  const float xi = Kpi[a] * Kqr[c] - Kpr[a] * Kqi[c] + Kqi[a] * Kpr[c] - Kqr[a] * Kpi[c];
                  const float hr = rec[4 + 2 * pr], hi = rec[5 + 2 * pr];
                  const int dl = P.pdelta[pr] - 1;
                  const float qr = hr * xr - hi * xi, qi = hr * xi + hi * xr;
#pragma unroll
                  for (int z = 0; z < 3; ++z)
                    if (z == dl) { Qr[z] += qr; Qi[z] += qi; }
                }
              float4 *cf = &T.hs[ja * PS_MAXPHI + (ja & 3) * 2 + r * 2];
              cf[0] = make_float4(Dc, Qr[0], Qr[1], Qr[2]);
              cf[1] = make_float4(Qi[0], Qi[1], Qi[2], 0.f);
            }
          }
          named_bar_sync(1, QEPT);
          // (b) every thread: its row's coefficients, then [hh]^+ / 2 on its 4 phases.
          // The entries' fourth words carry the row's polarisation factors for the
          // row pass: K_{s, c} (slot s, component c of (Re K+, Im K+, Re Kx, Im Kx))
          // in entry 4 s + c + (j & 1), so that the two rows a warp reads at once
          // (j even and odd) sit in different banks.
          const bool rowv = i < P.n_rows;
          const bool act = rowv && o0 < P.n_phi;
          float kw[4] = {0.f, 0.f, 0.f, 0.f};
          if (rowv) {
#pragma unroll
            for (int oo = 0; oo < 4; ++oo) {
              const int q = o0 + oo - (j & 1);
              if (q >= 0 && q < 4 * MAXM && ((P.slot_mask >> (q >> 2)) & 1u))
                kw[oo] = __ldg(reinterpret_cast<const float *>(P.pol) + (i * M + P.slot[q >> 2]) * 4 + (q & 3));
            }
          }
          float Dc[3] = {0.f, 0.f, 0.f}, Qr[3][3] = {}, Qi[3][3] = {};
          if (act) {
            const float4 *cf = &T.hs[j * PS_MAXPHI + (j & 3) * 2];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
              const float4 u0 = cf[2 * r], u1 = cf[2 * r + 1];
              Dc[r] = u0.x; Qr[r][0] = u0.y; Qr[r][1] = u0.z; Qr[r][2] = u0.w;
              Qi[r][0] = u1.x; Qi[r][1] = u1.y; Qi[r][2] = u1.z;
            }
          }
          named_bar_sync(1, QEPT);  // every row's coefficients read before T.hs is overwritten
          if (rowv) {
#pragma unroll
            for (int oo = 0; oo < 4; ++oo) {
              const int o = o0 + oo;
              if (!act) {
                T.hs[j * PS_MAXPHI + o] = make_float4(0.f, 0.f, 0.f, kw[oo]);
                continue;
              }
              float hh[3];
#pragma unroll
              for (int r = 0; r < 3; ++r) hh[r] = Dc[r];
#pragma unroll
              for (int dl = 0; dl < 3; ++dl) {
                const float2 e = T.phd[o * 3 + dl];
#pragma unroll
                for (int r = 0; r < 3; ++r) hh[r] += Qr[r][dl] * e.x - Qi[r][dl] * e.y;
              }
              const float A = hh[0], B = hh[1], C = hh[2];
              const float det = A * C - B * B;
              float a = 0.f, bb = 0.f, c = 0.f;
              if (det > P.rank_tol * A * C) {
                const float inv = 0.5f / det;
                a = C * inv; bb = -B * inv; c = A * inv;
              } else if (A > 0.f || C > 0.f) {
                const float sm = A + C;
                const float inv = 0.5f / (sm * sm);
                a = A * inv; bb = B * inv; c = C * inv;
              }
              // the accumulators' scale enters ln L^ML squared: fold it into the table
              T.hs[j * PS_MAXPHI + o] = make_float4(a * zs2, 2.f * bb * zs2, c * zs2, kw[oo]);
            }
          }
        }
      }
      named_bar_sync(1, QEPT);
      if (!mbar_wait(&T.tfull[b], use & 1, nullptr, abortp, P.wait_ns)) break;
      tc_fence_after();
      // ---- the rows: this lane's column, the warp's 16 rows
      const int t = c0 - k * P.n_tpad + (POL ? (L >> 2) : (L >> 1));
      const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + b * Q_BUF_COLS;
      const int j0 = sub * QJW;
      if constexpr (POL) {
        switch ((pair ? 8 : 0) + (pair ? P.n_even : 2)) {
          case 8: tile_rows_pol<0, 1>(P, T, tbase, rb, j0, k, t, part, lane, &T.tempty[b]); break;
          case 9: tile_rows_pol<1, 1>(P, T, tbase, rb, j0, k, t, part, lane, &T.tempty[b]); break;
          case 10: tile_rows_pol<2, 1>(P, T, tbase, rb, j0, k, t, part, lane, &T.tempty[b]); break;
          case 11: tile_rows_pol<3, 1>(P, T, tbase, rb, j0, k, t, part, lane, &T.tempty[b]); break;
          case 12: tile_rows_pol<4, 1>(P, T, tbase, rb, j0, k, t, part, lane, &T.tempty[b]); break;
          default: tile_rows_pol<2, 0>(P, T, tbase, rb, j0, k, t, part, lane, &T.tempty[b]); break;
        }
      } else {
        // a mode bank's azimuthal numbers are distinct in 1..4, one per class m mod 4:
        // quarter turns whenever n_phi % 4 == 0, else every phase on its own
        if (P.quad) tile_rows_modes<2>(P, T, tbase, rb, j0, k, t, part, lane, &T.tempty[b]);
        else tile_rows_modes<0>(P, T, tbase, rb, j0, k, t, part, lane, &T.tempty[b]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, Q_TMEM_COLS);
  if (threadIdx.x == 0 && T.abort_flag) atomicCAS(P.status, 0, DEV_E_TIMEOUT);
}

template <bool BF16, bool SPLIT, int VAR>
static cudaError_t launch_presel_variant(const CUtensorMap &mapG, const CUtensorMap &mapBank, const PreselParams &p,
                                         int grid, cudaStream_t st) {
  auto kern = presel_kernel<BF16, SPLIT, VAR>;
  const size_t smem = q_smem_bytes<SPLIT, VAR == 1>();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, QNT, smem, st>>>(mapG, mapBank, p);
  return cudaGetLastError();
}

template <int VAR>
static cudaError_t launch_presel_pm(const CUtensorMap &mapG, const CUtensorMap &mapBank, const PreselParams &p,
                                    bool bf16, bool split, int grid, cudaStream_t st) {
  if (bf16) return split ? launch_presel_variant<true, true, VAR>(mapG, mapBank, p, grid, st)
                         : launch_presel_variant<true, false, VAR>(mapG, mapBank, p, grid, st);
  return split ? launch_presel_variant<false, true, VAR>(mapG, mapBank, p, grid, st)
               : launch_presel_variant<false, false, VAR>(mapG, mapBank, p, grid, st);
}

}  // namespace dotpe
