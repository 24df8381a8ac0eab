// Fused per-pair epilogue shared by the FP32 SIMT and tcgen05 kernels.
//
// Given the per-mode components Z_m = sum_b h_{im}(b) G_m[b,e] of one (i,e)
// pair (Eq. dh_ieo: Re<d|h>(phi) = Re sum_m Z_m e^{i m phi}) and the <h|h>
// coefficients C_0, C_delta (Eq. hh_ieo: <h|h>(phi) = C_0 + 2 Re sum_delta
// C_delta e^{i delta phi}), evaluate on the regular phase grid phi_o:
//   ln L^ML_o   (Eq. bestfit_lnl),
//   the coherent-ML selection (Eq. coherent_ML_selection) against `thr`,
//   ln Lbar_o   (Eq. lnl_dist_marginalized, device table),
//   and the phase sums ln sum_o Lbar_o, ln sum_o Lbar_o^2 (w_o = 1).
#pragma once
#include "common.cuh"
#include "dist_marg.cuh"

namespace dotpe {

struct PairRes {
  float lsum;   // ln sum_o Lbar_o (-inf if no phase marginalised)
  float lsum2;  // ln sum_o Lbar_o^2
  float ml;     // max_o ln L^ML_o
  int argo;     // its phase index (lowest on ties)
  int npass;    // phases marginalised
};

// Phase tables in shared memory: ph_mode[m][o] = (cos, sin)(m_m phi_o) for the
// waveform's modes, ph_delta[k-1][o] = (cos, sin)(k phi_o), k = 1..3.
__device__ __forceinline__ void fill_phase_tables(float2 *ph, const EpiParams &P, int tid, int nthreads) {
  for (int k = tid; k < 7 * MAXPHI; k += nthreads) {
    int row = k / MAXPHI, o = k % MAXPHI;
    int mult = row < MAXM ? (row < P.n_modes ? P.mode_m[row] : 0) : (row - MAXM + 1);
    float s, c;
    // angle = mult * 2 pi o / n_phi, reduced exactly in integers first
    int num = (mult * o) % (P.n_phi > 0 ? P.n_phi : 1);
    sincospif(2.0f * (float)num / (float)P.n_phi, &s, &c);
    ph[k] = make_float2(c, s);
  }
}

// <h|h> coefficients for a polarisation-resolved bank (Eqs. hh_ieo with the
// polarisation index): H_{mm'} = sum_d sum_{pp'} F_p F_p' <h_{mp}|h_{m'p'}>_d.
// The row record of detector d (mrow + d REC_P, read through the cache) holds
// the overlaps grouped by delta = m - m': [X0, Y0, W0] for delta = 0 (real), then
// for delta = 1..3 (X, Y, W) complex, with X = sum <h_a+|h_c+>, Y = sum (<h_a+|h_cx>
// + <h_ax|h_c+>), W = sum <h_ax|h_cx>; the column record holds (F+^2, F+ Fx, Fx^2).
__device__ __forceinline__ void hh_coeffs_pol(const float *__restrict__ mrow, const float *__restrict__ qrec,
                                              const EpiParams &P, float &C0, float Cr[3], float Ci[3]) {
  C0 = 0.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) { Cr[k] = 0.f; Ci[k] = 0.f; }
  for (int d = 0; d < P.n_det; ++d) {
    const float *r = mrow + d * REC_P;
    const float *q = qrec + d * REC;
    const float q0 = q[0], q1 = q[1], q2 = q[2];
    C0 += q0 * __ldg(r) + q1 * __ldg(r + 1) + q2 * __ldg(r + 2);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float *g = r + 3 + 6 * k;
      Cr[k] += q0 * __ldg(g) + q1 * __ldg(g + 2) + q2 * __ldg(g + 4);
      Ci[k] += q0 * __ldg(g + 1) + q1 * __ldg(g + 3) + q2 * __ldg(g + 5);
    }
  }
}

// <h|h> coefficients for one pair from the row record (mrec) and column record (qrec):
// C_0 = sum_d sum_m M_d[m,m] Q_d[m,m];  C_delta = sum_d sum_{a>b, m_a-m_b=delta} M_d[a,b] Q_d[a,b].
// CONSEC: the modes' azimuthal numbers are consecutive, so pair (a, b) has delta = a - b.
// Each detector accumulates into its own partial sums (independent FMA chains),
// added at the end; records of detectors d >= n_det are zero.
// The row record's entry k of detector d is mr_at(d REC + k) (registers or memory).
template <bool CONSEC, class Row>
__device__ __forceinline__ void hh_coeffs_by(Row mr_at, const float *__restrict__ qrec, const EpiParams &P,
                                             float &C0, float Cr[3], float Ci[3]) {
  float c0[MAXD], cr[MAXD][3], ci[MAXD][3];
#pragma unroll
  for (int d = 0; d < MAXD; ++d) {
    c0[d] = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) { cr[d][k] = 0.f; ci[d][k] = 0.f; }
  }
  const int nd = P.n_det;
#pragma unroll
  for (int d = 0; d < MAXD; ++d) {
    if (d >= nd) break;
    auto mr = [&](int k) { return mr_at(d * REC + k); };
    const float4 *q4 = reinterpret_cast<const float4 *>(qrec + d * REC);
    float qr[REC];
#pragma unroll
    for (int v = 0; v < REC / 4; ++v) {
      const float4 x = q4[v];
      qr[4 * v] = x.x; qr[4 * v + 1] = x.y; qr[4 * v + 2] = x.z; qr[4 * v + 3] = x.w;
    }
#pragma unroll
    for (int m = 0; m < MAXM; ++m) c0[d] = fmaf(mr(m), qr[m], c0[d]);
    int p = 0;
#pragma unroll
    for (int a = 1; a < MAXM; ++a)
#pragma unroll
      for (int b = 0; b < a; ++b, ++p) {
        const float ar = mr(4 + 2 * p), ai = mr(5 + 2 * p);
        const float br = qr[4 + 2 * p], bi = qr[5 + 2 * p];
        if (CONSEC) {
          const int k = a - b - 1;
          cr[d][k] = fmaf(ar, br, fmaf(-ai, bi, cr[d][k]));
          ci[d][k] = fmaf(ar, bi, fmaf(ai, br, ci[d][k]));
        } else {
          const float hr = ar * br - ai * bi, hi = ar * bi + ai * br;
          const int dl = P.pdelta[p];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const bool sel = (dl == k + 1);
            cr[d][k] += sel ? hr : 0.f;
            ci[d][k] += sel ? hi : 0.f;
          }
        }
      }
  }
  C0 = (c0[0] + c0[1]) + c0[2];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    Cr[k] = (cr[0][k] + cr[1][k]) + cr[2][k];
    Ci[k] = (ci[0][k] + ci[1][k]) + ci[2][k];
  }
}

template <bool CONSEC>
__device__ __forceinline__ void hh_coeffs(const float *__restrict__ mrec, const float *__restrict__ qrec,
                                          const EpiParams &P, float &C0, float Cr[3], float Ci[3]) {
  hh_coeffs_by<CONSEC>([&](int k) { return mrec[k]; }, qrec, P, C0, Cr, Ci);
}

// Polarisation-resolved bank, row records held in registers (tensor-core
// epilogue): mrec [POL_TC_MAXD][REC_POL] as hh_coeffs_pol reads them from
// memory, the column record's (F+^2, F+ Fx, Fx^2) as one float4 per detector.
__device__ __forceinline__ void hh_coeffs_pol_reg(const float *mrec, const float *__restrict__ qrec,
                                                  const EpiParams &P, float &C0, float Cr[3], float Ci[3]) {
  C0 = 0.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) { Cr[k] = 0.f; Ci[k] = 0.f; }
#pragma unroll
  for (int d = 0; d < POL_TC_MAXD; ++d) {
    if (d >= P.n_det) break;
    const float4 q = *reinterpret_cast<const float4 *>(qrec + d * REC);
    const float *r = mrec + d * REC_POL;
    C0 += q.x * r[0] + q.y * r[1] + q.z * r[2];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      Cr[k] += q.x * r[3 + 6 * k] + q.y * r[5 + 6 * k] + q.z * r[7 + 6 * k];
      Ci[k] += q.x * r[4 + 6 * k] + q.y * r[6 + 6 * k] + q.z * r[8 + 6 * k];
    }
  }
}

// <h|h> coefficients of the tensor-core epilogue: HH = 0 general modes, 1
// consecutive modes, 2 polarisation-resolved bank (registers as above).
template <int HH>
__device__ __forceinline__ void hh_tile(const float *mrec, const float *__restrict__ qrec, const EpiParams &P,
                                        float &C0, float Cr[3], float Ci[3]) {
  if constexpr (HH == 2) hh_coeffs_pol_reg(mrec, qrec, P, C0, Cr, Ci);
  else hh_coeffs<HH == 1>(mrec, qrec, P, C0, Cr, Ci);
}

// Upper bound of max_o ln L^ML_o of a pair: |dh| <= sum_m |Z_m| and
// hh >= C_0 - 2 sum |C_delta| at every phase; +inf when that lower bound is not positive.
__device__ __forceinline__ float pair_bound(const float Zr[MAXM], const float Zi[MAXM], float C0, const float Cr[3],
                                            const float Ci[3]) {
  float a = 0.f, hmin = C0;
#pragma unroll
  for (int m = 0; m < MAXM; ++m) a += sqrtf(Zr[m] * Zr[m] + Zi[m] * Zi[m]);
#pragma unroll
  for (int k = 0; k < 3; ++k) hmin -= 2.f * sqrtf(Cr[k] * Cr[k] + Ci[k] * Ci[k]);
  return hmin > 0.f ? __fdividef(0.5f * a * a, hmin) * 1.000001f : INFINITY;
}

// Out-of-line distance marginal: it runs for the few phases that pass the ML
// cut, so it is kept out of the hot loop's instruction stream.
static __device__ __noinline__ float dm_lnlbar_call(float dh, float hh, float u_min, const float4 *tab) {
  return dm_lnlbar(dh, hh, u_min, tab);
}

__device__ __forceinline__ PairRes pair_eval(const float Zr[MAXM], const float Zi[MAXM], float C0,
                                             const float Cr[3], const float Ci[3], float thr, bool allow_skip,
                                             const EpiParams &P, const float2 *__restrict__ ph) {
  PairRes R;
  R.lsum = -INFINITY;
  R.lsum2 = -INFINITY;
  R.ml = 0.f;
  R.argo = 0;
  R.npass = 0;
  if (allow_skip && thr > 0.f) {
    // upper bound of max_o ln L^ML: |dh| <= sum |Z_m|, hh >= C_0 - 2 sum |C_delta|
    float a = 0.f, hmin = C0;
#pragma unroll
    for (int m = 0; m < MAXM; ++m) a += sqrtf(Zr[m] * Zr[m] + Zi[m] * Zi[m]);
#pragma unroll
    for (int k = 0; k < 3; ++k) hmin -= 2.f * sqrtf(Cr[k] * Cr[k] + Ci[k] * Ci[k]);
    if (hmin > 0.f && a * a < 2.f * hmin * thr) return R;
  }
  const float2 *phm = ph;
  const float2 *phd = ph + MAXM * MAXPHI;
  float mx = -INFINITY, s1 = 0.f, s2 = 0.f;
  float best = -1.f;
  int argo = 0, npass = 0;
#pragma unroll 2
  for (int o = 0; o < P.n_phi; ++o) {
    float dh = 0.f;
#pragma unroll
    for (int m = 0; m < MAXM; ++m) {
      float2 cs = phm[m * MAXPHI + o];
      dh = fmaf(Zr[m], cs.x, fmaf(-Zi[m], cs.y, dh));
    }
    float hs = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float2 cs = phd[k * MAXPHI + o];
      hs = fmaf(Cr[k], cs.x, fmaf(-Ci[k], cs.y, hs));
    }
    float hh = fmaf(2.f, hs, C0);
    float ml = (dh > 0.f && hh > 0.f) ? __fdividef(0.5f * dh * dh, hh) : 0.f;
    if (ml > best) { best = ml; argo = o; }
    if (!(ml >= thr)) continue;
    ++npass;
    float l = dm_lnlbar_call(dh, hh, P.u_min, P.dm_table);
    if (l > mx) {
      float r = __expf(mx - l);
      s1 = fmaf(s1, r, 1.f);
      s2 = fmaf(s2, r * r, 1.f);
      mx = l;
    } else {
      float q = __expf(l - mx);
      s1 += q;
      s2 = fmaf(q, q, s2);
    }
  }
  R.ml = best;
  R.argo = argo;
  R.npass = npass;
  if (npass > 0) {
    R.lsum = mx + __logf(s1);
    R.lsum2 = 2.f * mx + __logf(s2);
  }
  return R;
}

// Screening evaluation (no distance marginal): max_o ln L^ML_o and its phase.
// A pair whose upper bound (as in pair_eval) is below thr returns ml = -1: it
// cannot reach the cut.
__device__ __forceinline__ float pair_ml(const float Zr[MAXM], const float Zi[MAXM], float C0, const float Cr[3],
                                         const float Ci[3], float thr, bool allow_skip, const EpiParams &P,
                                         const float2 *__restrict__ ph, int &argo) {
  argo = 0;
  if (allow_skip && thr > 0.f) {
    float a = 0.f, hmin = C0;
#pragma unroll
    for (int m = 0; m < MAXM; ++m) a += sqrtf(Zr[m] * Zr[m] + Zi[m] * Zi[m]);
#pragma unroll
    for (int k = 0; k < 3; ++k) hmin -= 2.f * sqrtf(Cr[k] * Cr[k] + Ci[k] * Ci[k]);
    if (hmin > 0.f && a * a < 2.f * hmin * thr) return -1.f;
  }
  const float2 *phm = ph;
  const float2 *phd = ph + MAXM * MAXPHI;
  float best = -1.f;
#pragma unroll 4
  for (int o = 0; o < P.n_phi; ++o) {
    float dh = 0.f;
#pragma unroll
    for (int m = 0; m < MAXM; ++m) {
      float2 cs = phm[m * MAXPHI + o];
      dh = fmaf(Zr[m], cs.x, fmaf(-Zi[m], cs.y, dh));
    }
    float hs = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float2 cs = phd[k * MAXPHI + o];
      hs = fmaf(Cr[k], cs.x, fmaf(-Ci[k], cs.y, hs));
    }
    float hh = fmaf(2.f, hs, C0);
    float ml = (dh > 0.f && hh > 0.f) ? __fdividef(0.5f * dh * dh, hh) : 0.f;
    if (ml > best) { best = ml; argo = o; }
  }
  return best;
}

// Cut threshold of a tile (Eq. coherent_ML_selection): running maximum - cut_delta,
// lowered by twice the screening margin in a screening pass (so that no pair the
// exact product would keep is skipped); -inf when the cut is off.
__device__ __forceinline__ float tile_threshold(const EpiParams &P) {
  if (!(P.cut_delta > 0.f)) return -INFINITY;
  const float run = *(volatile float *)P.ml_running;
  float thr = run - P.cut_delta;
  if (P.margin_k > 0.f) thr -= 2.f * screen_margin(run, P.margin_k, *P.sqrt_dd);
  return thr;
}

// Online log-sum-exp accumulator.
struct Lse {
  float m, s;
  __device__ __forceinline__ void init() { m = -INFINITY; s = 0.f; }
  __device__ __forceinline__ void add(float x) {
    if (x == -INFINITY) return;
    if (x > m) { s = fmaf(s, __expf(m - x), 1.f); m = x; }
    else s += __expf(x - m);
  }
  __device__ __forceinline__ void merge(float om, float os) {
    if (om == -INFINITY) return;
    if (m == -INFINITY) { m = om; s = os; return; }
    if (om > m) { s = fmaf(s, __expf(m - om), os); m = om; }
    else s = fmaf(os, __expf(om - m), s);
  }
};

__device__ __forceinline__ void warp_merge_lse(Lse &a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float om = __shfl_xor_sync(0xffffffffu, a.m, o);
    float os = __shfl_xor_sync(0xffffffffu, a.s, o);
    a.merge(om, os);
  }
}

// (value, packed index) max with lowest index on ties
__device__ __forceinline__ void warp_argmax(float &v, long long &idx) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float ov = __shfl_xor_sync(0xffffffffu, v, o);
    long long oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
}

}  // namespace dotpe
