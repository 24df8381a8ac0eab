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

// Grid: ln s in [-12, 6] (step 1/8); y in [-64, 64], piecewise uniform: step 1/8 on
// [-64, -2] and [12, 64], 1/32 on [-2, 12] where, for small s, K switches over a width
// ~1/y between the far-distance term (s^-3 e^{-y^2/2}) and the peak term (y^-4).
constexpr float DM_YA = -64.0f, DM_YB = -2.0f, DM_YC = 12.0f, DM_YD = 64.0f;
constexpr float DM_HA = 0.125f, DM_HB = 0.03125f, DM_HC = 0.125f;
constexpr int DM_NA = 496, DM_NB = 448, DM_NC = 416;  // cells per segment
constexpr int DM_NY = DM_NA + DM_NB + DM_NC + 1;      // nodes
constexpr float DM_S0 = -12.0f, DM_DS = 0.125f;
constexpr int DM_NS = 145;
constexpr float DM_HH_FLOOR = 1e-30f;

// node index -> y (host and device, exact in binary)
__host__ __device__ __forceinline__ double dm_node_y(int iy) {
  if (iy <= DM_NA) return (double)DM_YA + (double)DM_HA * iy;
  if (iy <= DM_NA + DM_NB) return (double)DM_YB + (double)DM_HB * (iy - DM_NA);
  return (double)DM_YC + (double)DM_HC * (iy - DM_NA - DM_NB);
}

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

// K(y, sigma) from the table: float4 = (K, dK/dy, dK/dsigma * ds, d2K/dy dsigma * ds);
// the y-derivatives are scaled by the step of the cell being interpolated.
__device__ __forceinline__ float dm_table_K(float y, float sig, const float4 *__restrict__ tab) {
  float yscale = 1.0f;
  if (y < DM_YA) {
    // t ~ N(y, 1) truncated at 0 is exponential with rate |y| for y << 0, and then
    // K depends on |y| s only: move to the grid edge at equal |y| s
    sig += __logf(y * (1.0f / DM_YA));
    y = DM_YA;
  } else if (y > DM_YD) {
    // beyond the grid K ~ 10 Var(t) / (s + mu)^2: rescale from the last column
    float s = __expf(sig);
    float a = (s + dm_mu(DM_YD)) / (s + dm_mu(y));
    yscale = a * a;
    y = DM_YD;
  }
  float ext = 0.0f;  // linear extrapolation below the sigma grid
  float fs = (sig - DM_S0) * (1.0f / DM_DS);
  if (fs < 0.0f) {
    ext = fs;
    fs = 0.0f;
  }
  fs = fminf(fs, (float)(DM_NS - 1) - 1e-3f);
  int iy;
  float u, hy;
  if (y < DM_YB) {
    float f = (y - DM_YA) * (1.0f / DM_HA);
    iy = min(max((int)f, 0), DM_NA - 1);
    u = f - (float)iy;
    hy = DM_HA;
  } else if (y < DM_YC) {
    float f = (y - DM_YB) * (1.0f / DM_HB);
    int c = min(max((int)f, 0), DM_NB - 1);
    u = f - (float)c;
    iy = DM_NA + c;
    hy = DM_HB;
  } else {
    float f = (y - DM_YC) * (1.0f / DM_HC);
    int c = min(max((int)f, 0), DM_NC - 1);
    u = f - (float)c;
    iy = DM_NA + DM_NB + c;
    hy = DM_HC;
  }
  u = fminf(fmaxf(u, 0.0f), 1.0f);
  int is = (int)fs;
  float v = fs - (float)is;
  const float4 q00 = __ldg(&tab[is * DM_NY + iy]);
  const float4 q10 = __ldg(&tab[is * DM_NY + iy + 1]);
  const float4 q01 = __ldg(&tab[(is + 1) * DM_NY + iy]);
  const float4 q11 = __ldg(&tab[(is + 1) * DM_NY + iy + 1]);
  float a0, a1, b0, b1, c0, c1, d0, d1;
  hermite_basis(u, a0, b0, a1, b1);  // a0=h00(u) b0=h10(u) a1=h01(u) b1=h11(u)
  hermite_basis(v, c0, d0, c1, d1);
  b0 *= hy;
  b1 *= hy;
  float val = q00.x * a0 * c0 + q10.x * a1 * c0 + q01.x * a0 * c1 + q11.x * a1 * c1 +
              q00.y * b0 * c0 + q10.y * b1 * c0 + q01.y * b0 * c1 + q11.y * b1 * c1 +
              q00.z * a0 * d0 + q10.z * a1 * d0 + q01.z * a0 * d1 + q11.z * a1 * d1 +
              q00.w * b0 * d0 + q10.w * b1 * d0 + q01.w * b0 * d1 + q11.w * b1 * d1;
  if (ext != 0.0f) {
    // sigma-derivative at the lower edge, interpolated in y
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
  const float sig = __logf(s);  // ln s
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
