// Distance marginalisation (paper Eq. lnl_dist_marginalized) on the device.
//
// With pi(d_L) = 3 d_L^2 / d_max^3 on (0, d_max] and u = d_L^0 / d_L, the
// marginal likelihood of a phase with inner products (dh, hh) at d_L^0 is
//   Lbar = 3 u_min^3 int_{u_min}^inf u^-4 exp(dh u - hh u^2 / 2) du.
// With x = dh / sqrt(hh), s = u_min sqrt(hh), y = x - s and t = v - s:
//   ln Lbar = x^2/2 + ln 3 + 3 ln s + ln int_0^inf (s + t)^-4 e^{-(t - y)^2/2} dt
//           = x^2/2 + ln Phi(y) + ln 3 + (1/2) ln 2pi + 3 ln s
//             + ln E[(s + t)^-4],   t ~ N(y, 1) truncated to t >= 0.
// The first two terms carry the whole dynamic range and are evaluated
// analytically (erfc / erfcx).  The remainder is written as
//   ln E[(s + t)^-4] = -4 ln(s + mu(y)) + K(y, ln s),  mu(y) = (y + sqrt(y^2 + 4)) / 2,
// where mu tracks the mean of the truncated normal (-> y for y >> 0, -> 1/|y|
// for y << 0), which leaves K small and smooth.  K is tabulated on a regular
// (y, ln s) grid with its first and mixed derivatives (FP64 Gauss-Legendre,
// built once per context) and read back by bicubic Hermite interpolation.
#pragma once
#include "common.cuh"

namespace dotpe {

// Grid: y in [-40, 64], ln s in [-12, 6], steps of 1/8.
constexpr float DM_Y0 = -40.0f, DM_DY = 0.125f;
constexpr int DM_NY = 833;
constexpr float DM_S0 = -12.0f, DM_DS = 0.125f;
constexpr int DM_NS = 145;
constexpr float DM_HH_FLOOR = 1e-30f;

__device__ __forceinline__ float dm_mu(float y) {
  float r = sqrtf(fmaf(y, y, 4.0f));
  return y >= 0.0f ? 0.5f * (y + r) : 2.0f / (r - y);
}

__device__ __forceinline__ void hermite_basis(float t, float &h00, float &h10, float &h01, float &h11) {
  float t2 = t * t, omt = 1.0f - t;
  h00 = (1.0f + 2.0f * t) * omt * omt;
  h10 = t * omt * omt;
  h01 = t2 * (3.0f - 2.0f * t);
  h11 = t2 * (t - 1.0f);
}

// K(y, sigma) from the table (float4 = value, d/dy*dy, d/dsig*ds, d2/dy dsig*dy*ds).
__device__ __forceinline__ float dm_table_K(float y, float sig, const float4 *__restrict__ tab) {
  float ext = 0.0f;  // linear extrapolation below the sigma grid
  float fs = (sig - DM_S0) * (1.0f / DM_DS);
  if (fs < 0.0f) {
    ext = fs;  // in units of the grid step, times the sigma-derivative at the edge
    fs = 0.0f;
  }
  fs = fminf(fs, (float)(DM_NS - 1) - 1e-3f);
  float fy = (y - DM_Y0) * (1.0f / DM_DY);
  float yscale = 1.0f;
  if (fy > (float)(DM_NY - 1)) {
    // beyond the grid K ~ 10 Var(t) / (s + mu)^2: rescale from the last column
    float ylast = DM_Y0 + DM_DY * (float)(DM_NY - 1);
    float s = __expf(sig);
    float a = (s + dm_mu(ylast)) / (s + dm_mu(y));
    yscale = a * a;
    fy = (float)(DM_NY - 1) - 1e-3f;
  }
  fy = fmaxf(fy, 0.0f);
  int iy = (int)fy, is = (int)fs;
  float u = fy - (float)iy, v = fs - (float)is;
  const float4 q00 = __ldg(&tab[is * DM_NY + iy]);
  const float4 q10 = __ldg(&tab[is * DM_NY + iy + 1]);
  const float4 q01 = __ldg(&tab[(is + 1) * DM_NY + iy]);
  const float4 q11 = __ldg(&tab[(is + 1) * DM_NY + iy + 1]);
  float a0, a1, b0, b1, c0, c1, d0, d1;
  hermite_basis(u, a0, b0, a1, b1);  // a0=h00(u) b0=h10(u) a1=h01(u) b1=h11(u)
  hermite_basis(v, c0, d0, c1, d1);
  float val = q00.x * a0 * c0 + q10.x * a1 * c0 + q01.x * a0 * c1 + q11.x * a1 * c1 +
              q00.y * b0 * c0 + q10.y * b1 * c0 + q01.y * b0 * c1 + q11.y * b1 * c1 +
              q00.z * a0 * d0 + q10.z * a1 * d0 + q01.z * a0 * d1 + q11.z * a1 * d1 +
              q00.w * b0 * d0 + q10.w * b1 * d0 + q01.w * b0 * d1 + q11.w * b1 * d1;
  if (ext != 0.0f) {
    // sigma-derivative at the lower edge, interpolated in y (Hermite in u)
    float dsv = q00.z * a0 + q10.z * a1 + q00.w * b0 + q10.w * b1;
    val += ext * dsv;
  }
  return val * yscale;
}

// ln Lbar(dh, hh) for d_L^0 / d_max = u_min.  hh <= floor: no signal power -> 0.
__device__ __forceinline__ float dm_lnlbar(float dh, float hh, float u_min, const float4 *__restrict__ tab) {
  if (!(hh > DM_HH_FLOOR)) return 0.0f;
  const float r = sqrtf(hh);
  const float x = dh / r;
  const float s = u_min * r;
  const float y = x - s;
  const float sig = __logf(s);
  const float RS2 = 0.70710678118654752f;
  float base;  // x^2/2 + ln Phi(y)
  if (y >= 0.0f) {
    base = 0.5f * x * x + log1pf(-0.5f * erfcf(y * RS2));
  } else {
    base = s * (x - 0.5f * s) + __logf(0.5f * erfcxf(-y * RS2));
  }
  const float C = 2.0175508218727822f;  // ln 3 + ln(2 pi)/2
  return base + C + 3.0f * sig - 4.0f * __logf(s + dm_mu(y)) + dm_table_K(y, sig, tab);
}

}  // namespace dotpe
