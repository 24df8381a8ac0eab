// Per-event preparation, bank conversion and the distance-marginal table.
//
//  K0  prep_bins / prep_ext   data weights c_{d,b} = 4 w_b conj(d_d(f_b)) / S_d(f_b) and
//                             omega_{d,b} = 4 w_b / S_d(f_b) (Eq. inner_product) in FP64,
//                             input validation, FP32 hi/lo splits of f and t
//  K1  build_G / pack_G       G_m[b,e] = sum_d R_{e,d,m} exp(-2 pi i f_b t_{e,d}) c_{d,b}
//                             (Eq. dh_ieo with the detector sum folded into G), packed as
//                             the real-ified K-major operand [(e,re),(e,im)] x [re | im];
//                             column cross-term records Q_d[e] = R_{e,d,m} R^*_{e,d,m'}
//                             (Eq. hh_ieo)
//  K2  cross_terms            row records <h_{im}|h_{im'}>_d = sum_b omega_{d,b} h h'^*
//  K9  build_dm_table         FP64 Gauss-Legendre table of the distance-marginal remainder
#include <cstdio>
#include <mutex>
#include <type_traits>

#include "common.cuh"
#include "dist_marg.cuh"
#include "kernels.h"

namespace dotpe {

// ---------------------------------------------------------------------------
// K0
// ---------------------------------------------------------------------------
// Data weights of every component j (a mode, or a (mode, polarisation) pair
// j = 2m + p of a polarisation-resolved bank; M counts components here),
// c[d][j][b]: the plain quadrature's 4 w_b conj(d_d(f_b)) / S_d(f_b) (the same
// for every component), or, with relative binning (App. A, Eqs. dh_weights,
// d_h), conj(W^{<d|h>}_{d j b}).
__global__ void prep_bins_kernel(int D, int B, int M, const double *__restrict__ f, const double *__restrict__ w,
                                 const double *__restrict__ psd, const double2 *__restrict__ data,
                                 const double2 *__restrict__ rb_dh, float2 *__restrict__ c,
                                 float *__restrict__ omega, float *__restrict__ fh, float *__restrict__ fl,
                                 int *status) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < B) {
    double fb = f[k];
    float h = (float)fb;
    fh[k] = h;
    fl[k] = (float)(fb - (double)h);
    if (!isfinite(fb) || !isfinite(w[k])) atomicCAS(status, 0, DEV_E_NONFINITE);
  }
  if (k >= D * B) return;
  const int b = k % B, d = k / B;
  if (rb_dh) {
    omega[k] = 0.f;
    for (int m = 0; m < M; ++m) {
      double2 v = rb_dh[((int64_t)d * M + m) * B + b];
      if (!isfinite(v.x) || !isfinite(v.y)) { atomicCAS(status, 0, DEV_E_NONFINITE); v = make_double2(0.0, 0.0); }
      c[((int64_t)d * M + m) * B + b] = make_float2((float)v.x, (float)(-v.y));
    }
    return;
  }
  double S = psd[k];
  double2 dk = data[k];
  if (!(S > 0.0) || !isfinite(S) || !isfinite(dk.x) || !isfinite(dk.y)) {
    atomicCAS(status, 0, DEV_E_NONFINITE);
    S = 1.0; dk = make_double2(0.0, 0.0);
  }
  double om = 4.0 * w[b] / S;
  omega[k] = (float)om;
  const float2 cv = make_float2((float)(om * dk.x), (float)(-om * dk.y));
  for (int m = 0; m < M; ++m) c[((int64_t)d * M + m) * B + b] = cv;
}

// Relative binning: the Cauchy-Schwarz scale of the screening margin,
// sqrt(max_m sum_{d,b} |W^{<d|h>}_{d m b}|^2 / W^{<h|h>}_{d m m b}) (with plain
// weights the same sum is <d|d>), in FP64, one block, fixed order.
__global__ void rb_norm_kernel(int D, int M, int B, const double2 *__restrict__ rb_dh,
                               const double2 *__restrict__ rb_hh, float *__restrict__ sqrt_dd) {
  __shared__ double part[256];
  double best = 0.0;
  for (int m = 0; m < M; ++m) {
    double v = 0.0;
    for (int k = threadIdx.x; k < D * B; k += blockDim.x) {
      const int d = k / B, b = k % B;
      const double2 a = rb_dh[((int64_t)d * M + m) * B + b];
      const double h = rb_hh[(((int64_t)d * M + m) * M + m) * B + b].x;
      if (h > 0.0 && isfinite(h)) v += (a.x * a.x + a.y * a.y) / h;
    }
    part[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
      __syncthreads();
    }
    best = fmax(best, part[0]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *sqrt_dd = (float)sqrt(best);
}

// sqrt<d|d> = sqrt(sum_{d,b} omega_{d,b} |d_d(f_b)|^2) in FP64, one block, fixed order.
__global__ void data_norm_kernel(int D, int B, const double *__restrict__ w, const double *__restrict__ psd,
                                 const double2 *__restrict__ data, float *__restrict__ sqrt_dd) {
  __shared__ double part[256];
  double v = 0.0;
  for (int k = threadIdx.x; k < D * B; k += blockDim.x) {
    const double S = psd[k];
    const double2 dk = data[k];
    if (S > 0.0 && isfinite(S) && isfinite(dk.x) && isfinite(dk.y)) v += 4.0 * w[k % B] / S * (dk.x * dk.x + dk.y * dk.y);
  }
  part[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *sqrt_dd = (float)sqrt(part[0]);
}

// F non-null (polarisation-resolved bank): the column record is (F+^2, F+ Fx, Fx^2)
// of the real antenna patterns F [E][D][2] and R is not read.
__global__ void prep_ext_kernel(int64_t E, int D, int M, const double *__restrict__ t,
                                const double2 *__restrict__ R, const double *__restrict__ F,
                                float *__restrict__ th, float *__restrict__ tl,
                                float2 *__restrict__ Rf, float *__restrict__ qx, int *status) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= E * D) return;
  double tv = t[k];
  if (!isfinite(tv)) { atomicCAS(status, 0, DEV_E_NONFINITE); tv = 0.0; }
  float h = (float)tv;
  th[k] = h;
  tl[k] = (float)(tv - (double)h);
  if (F) {
    double fp = F[2 * k], fx = F[2 * k + 1];
    if (!isfinite(fp) || !isfinite(fx)) { atomicCAS(status, 0, DEV_E_NONFINITE); fp = 0.0; fx = 0.0; }
    float *q = qx + k * REC;
    q[0] = (float)(fp * fp);
    q[1] = (float)(fp * fx);
    q[2] = (float)(fx * fx);
    for (int j = 3; j < REC; ++j) q[j] = 0.f;
    return;
  }
  float2 r[MAXM];
#pragma unroll
  for (int m = 0; m < MAXM; ++m) {
    double2 v = (m < M) ? R[k * M + m] : make_double2(0.0, 0.0);
    if (!isfinite(v.x) || !isfinite(v.y)) { atomicCAS(status, 0, DEV_E_NONFINITE); v = make_double2(0.0, 0.0); }
    r[m] = make_float2((float)v.x, (float)v.y);
    if (m < M) Rf[k * M + m] = r[m];
  }
  // column record of <h|h>: |R_m|^2 and R_a R_b^* for a > b (Eq. hh_ieo)
  float *q = qx + k * REC;
#pragma unroll
  for (int m = 0; m < MAXM; ++m) q[m] = r[m].x * r[m].x + r[m].y * r[m].y;
  int p = 0;
#pragma unroll
  for (int a = 1; a < MAXM; ++a)
#pragma unroll
    for (int b = 0; b < a; ++b, ++p) {
      q[4 + 2 * p] = r[a].x * r[b].x + r[a].y * r[b].y;
      q[5 + 2 * p] = r[a].y * r[b].x - r[a].x * r[b].y;
    }
}

// ---------------------------------------------------------------------------
// K1
// ---------------------------------------------------------------------------
// exp(-2 pi i f t) with the phase f t formed to ~1e-9 cycles in FP32:
// exact product of the hi parts (FMA), cross terms of the lo parts.
__device__ __forceinline__ float2 shift_factor(float fh, float fl, float th, float tl) {
  float p = fh * th;
  float e1 = fmaf(fh, th, -p);
  float e2 = fmaf(fh, tl, fl * th);
  float n = rintf(p);
  float q = (p - n) + (e1 + e2);
  float s, c;
  sincospif(2.0f * q, &s, &c);
  return make_float2(c, -s);
}

__global__ void build_G_kernel(int64_t E, int D, int M, int B, const float *__restrict__ fh,
                               const float *__restrict__ fl, const float *__restrict__ th,
                               const float *__restrict__ tl, const float2 *__restrict__ c,
                               const float2 *__restrict__ Rf, float2 *__restrict__ G /*[M][E][B]*/,
                               float *__restrict__ gmax) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= E * B) return;
  int64_t e = k / B;
  int b = (int)(k % B);
  float2 g[MAXM];
#pragma unroll
  for (int m = 0; m < MAXM; ++m) g[m] = make_float2(0.f, 0.f);
  float f_h = fh[b], f_l = fl[b];
  for (int d = 0; d < D; ++d) {
    float2 T = shift_factor(f_h, f_l, th[e * D + d], tl[e * D + d]);
#pragma unroll
    for (int m = 0; m < MAXM; ++m) {
      if (m >= M) break;
      const float2 cc = c[((int64_t)d * M + m) * B + b];
      const float2 W = make_float2(T.x * cc.x - T.y * cc.y, T.x * cc.y + T.y * cc.x);
      float2 r = Rf[(e * D + d) * M + m];
      g[m].x += r.x * W.x - r.y * W.y;
      g[m].y += r.x * W.y + r.y * W.x;
    }
  }
  float a = 0.f;
#pragma unroll
  for (int m = 0; m < MAXM; ++m) {
    if (m >= M) break;
    G[((int64_t)m * E + e) * B + b] = g[m];
    a = fmaxf(a, fmaxf(fabsf(g[m].x), fabsf(g[m].y)));
  }
  atomic_max_nonneg(gmax, a);
}

// Polarisation-resolved bank: G_{m p}[b, e] = sum_d F_{e d p} e^{-2 pi i f_b t_{e d}} c_{d m p b},
// G [M][2][E][B] (Eq. dh_ieo with the polarisation index; real antenna patterns); the data
// weights c [D][M][2][B] are per component (the same for both with plain quadrature).
__global__ void build_G_pol_kernel(int64_t E, int D, int M, int B, const float *__restrict__ fh,
                                   const float *__restrict__ fl, const float *__restrict__ th,
                                   const float *__restrict__ tl, const float2 *__restrict__ c,
                                   const double *__restrict__ F, float2 *__restrict__ G,
                                   float *__restrict__ gmax) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= E * B) return;
  int64_t e = k / B;
  int b = (int)(k % B);
  float2 g[MAXM][2];
#pragma unroll
  for (int m = 0; m < MAXM; ++m) { g[m][0] = make_float2(0.f, 0.f); g[m][1] = make_float2(0.f, 0.f); }
  float f_h = fh[b], f_l = fl[b];
  for (int d = 0; d < D; ++d) {
    const float2 T = shift_factor(f_h, f_l, th[e * D + d], tl[e * D + d]);
    const float fp = (float)F[(e * D + d) * 2], fx = (float)F[(e * D + d) * 2 + 1];
#pragma unroll
    for (int m = 0; m < MAXM; ++m) {
      if (m >= M) break;
      const float2 c0 = c[((int64_t)(d * M + m) * 2) * B + b], c1 = c[((int64_t)(d * M + m) * 2 + 1) * B + b];
      const float2 W0 = make_float2(T.x * c0.x - T.y * c0.y, T.x * c0.y + T.y * c0.x);
      const float2 W1 = make_float2(T.x * c1.x - T.y * c1.y, T.x * c1.y + T.y * c1.x);
      g[m][0].x += fp * W0.x; g[m][0].y += fp * W0.y;
      g[m][1].x += fx * W1.x; g[m][1].y += fx * W1.y;
    }
  }
  float a = 0.f;
#pragma unroll
  for (int m = 0; m < MAXM; ++m) {
    if (m >= M) break;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      G[(((int64_t)m * 2 + q) * E + e) * B + b] = g[m][q];
      a = fmaxf(a, fmaxf(fabsf(g[m][q].x), fabsf(g[m][q].y)));
    }
  }
  atomic_max_nonneg(gmax, a);
}

// fp16 operands are scaled to magnitudes up to 2^14 instead of 1: the five
// exponent bits then keep hi normal down to ~4e-9 of the largest element and lo
// (~2^-11 hi) normal down to ~8e-6 of it, so the split keeps ~2^-22 relative
// accuracy over the data's dynamic range (products and K-sums stay far inside FP32).
__device__ __forceinline__ float pow2_scale(float maxabs) {
  // 2^-ceil(log2(maxabs)): scaled magnitudes land in (1/2, 1]
  if (!(maxabs > 0.f) || !isfinite(maxabs)) return 1.0f;
  int ex;
  frexpf(maxabs, &ex);
  return ldexpf(1.0f, -ex);
}

// Real-ified operand rows: (e, re) = [Gr | -Gi], (e, im) = [Gi | Gr], K padded with zeros
// (the bank rows use the same column order: [Re h | Im h | 0]).
// kind: 0 = fp32 plane, 1 = bf16 hi, 2 = fp16 hi; nplanes == 2 adds the lo plane
// RN(v - hi) of the same type.  One thread per (m, e, c): for c < B it reads
// G[m][e][c] once and writes the four entries that hold it (columns c and B + c
// of both rows); for c < Kpad - 2B it zeroes column 2B + c of both rows.
template <typename T>
__device__ __forceinline__ void put(void *out, int64_t total, int64_t k, float v, int nplanes) {
  if constexpr (sizeof(T) == 4) {
    ((float *)out)[k] = v;
  } else {
    T hi;
    float hf;
    if constexpr (std::is_same<T, __nv_bfloat16>::value) { hi = __float2bfloat16_rn(v); hf = __bfloat162float(hi); }
    else { hi = __float2half_rn(v); hf = __half2float(hi); }
    ((T *)out)[k] = hi;
    if (nplanes == 2) {
      if constexpr (std::is_same<T, __nv_bfloat16>::value) ((T *)out)[total + k] = __float2bfloat16_rn(v - hf);
      else ((T *)out)[total + k] = __float2half_rn(v - hf);
    }
  }
}

template <typename T>
__global__ void pack_G_kernel(int64_t E, int M, int B, int Kpad, int NP, const float2 *__restrict__ G,
                              const float *__restrict__ gmax, int kind, int nplanes, void *__restrict__ out,
                              float *__restrict__ scale_out) {
  // NP polarisation blocks along K (1, or 2 for a polarisation-resolved bank):
  // row (m, e, re) = [Gr_0 | -Gi_0 | Gr_1 | -Gi_1 | 0], (m, e, im) = [Gi_0 | Gr_0 | Gi_1 | Gr_1 | 0]
  const int pad = Kpad - 2 * NP * B;
  const int P = B > pad ? B : pad;  // threads per (m, e)
  const int64_t total = (int64_t)M * 2 * E * Kpad;
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const float sc = (kind == 0) ? 1.0f : pow2_scale(*gmax) * (kind == 2 ? FP16_OPERAND_SCALE : 1.0f);
  if (k == 0 && scale_out) *scale_out = sc;
  if (k >= (int64_t)M * E * P) return;
  const int c = (int)(k % P);
  const int64_t me = k / P;  // m * E + e
  const int64_t m = me / E, e = me - m * E;
  // element (part, column) of sample me: the 16-bit planes keep the two rows
  // [2 me][Kpad] and [2 me + 1][Kpad] (tensor-core B rows); the FP32 operand of
  // the CUDA-core kernel interleaves them, [me][Kpad][2] = (re row, im row) per column
  auto at = [&](int part, int64_t col) -> int64_t {
    if constexpr (sizeof(T) == 4) return (me * Kpad + col) * 2 + part;
    else return (2 * me + part) * Kpad + col;
  };
  if (c < B) {
    for (int q = 0; q < NP; ++q) {
      const float2 g = G[((m * NP + q) * E + e) * B + c];
      const float gr = g.x * sc, gi = g.y * sc;
      const int o = 2 * q * B;
      put<T>(out, total, at(0, o + c), gr, nplanes);
      put<T>(out, total, at(0, o + B + c), -gi, nplanes);
      put<T>(out, total, at(1, o + c), gi, nplanes);
      put<T>(out, total, at(1, o + B + c), gr, nplanes);
    }
  }
  if (c < pad) {
    put<T>(out, total, at(0, 2 * NP * B + c), 0.f, nplanes);
    put<T>(out, total, at(1, 2 * NP * B + c), 0.f, nplanes);
  }
}

// ---------------------------------------------------------------------------
// K2: row records <h_{im}|h_{im'}>_d  (one warp per bank row)
// ---------------------------------------------------------------------------
// RB: the weight of each mode pair is W^{<h|h>}_{d a c b} of relative binning
// (App. A, Eq. h_h; complex, rb_hh [D][M][M][B]) instead of omega_{d b}.
template <bool RB>
__global__ void cross_terms_kernel(int64_t n_rows, int64_t row0, int64_t I_bank, int M, int D, int B, int Kpad,
                                   const float *__restrict__ master /*[M][I_bank][Kpad]*/,
                                   const float *__restrict__ omega /*[D][B]*/,
                                   const double2 *__restrict__ rb_hh, float *__restrict__ mx) {
  extern __shared__ float om_s[];
  if (!RB)
    for (int k = threadIdx.x; k < D * B; k += blockDim.x) om_s[k] = omega[k];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warp_global = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp_global; i < n_rows; i += nwarps) {
    float acc[MAXD][REC];
#pragma unroll
    for (int d = 0; d < MAXD; ++d)
#pragma unroll
      for (int q = 0; q < REC; ++q) acc[d][q] = 0.f;
    for (int b = lane; b < B; b += 32) {
      float hr[MAXM], hi[MAXM];
#pragma unroll
      for (int m = 0; m < MAXM; ++m) {
        if (m < M) {
          const float *row = master + ((int64_t)m * I_bank + row0 + i) * Kpad;
          hr[m] = __ldg(row + b);
          hi[m] = __ldg(row + B + b);
        } else {
          hr[m] = 0.f; hi[m] = 0.f;
        }
      }
#pragma unroll
      for (int d = 0; d < MAXD; ++d) {
        if (d >= D) break;
        if (!RB) {
          float w = om_s[d * B + b];
#pragma unroll
          for (int m = 0; m < MAXM; ++m) acc[d][m] += w * (hr[m] * hr[m] + hi[m] * hi[m]);
          int p = 0;
#pragma unroll
          for (int a = 1; a < MAXM; ++a)
#pragma unroll
            for (int c = 0; c < a; ++c, ++p) {
              // h_a h_c^*
              acc[d][4 + 2 * p] += w * (hr[a] * hr[c] + hi[a] * hi[c]);
              acc[d][5 + 2 * p] += w * (hi[a] * hr[c] - hr[a] * hi[c]);
            }
        } else {
#pragma unroll
          for (int m = 0; m < MAXM; ++m) {
            if (m >= M) break;
            const float w = (float)__ldg(&rb_hh[(((int64_t)d * M + m) * M + m) * B + b].x);
            acc[d][m] += w * (hr[m] * hr[m] + hi[m] * hi[m]);
          }
          int p = 0;
#pragma unroll
          for (int a = 1; a < MAXM; ++a)
#pragma unroll
            for (int c = 0; c < a; ++c, ++p) {
              if (a >= M) continue;
              const double2 wv = __ldg(&rb_hh[(((int64_t)d * M + a) * M + c) * B + b]);
              const float wr = (float)wv.x, wi = (float)wv.y;
              const float pr = hr[a] * hr[c] + hi[a] * hi[c], pi = hi[a] * hr[c] - hr[a] * hi[c];
              acc[d][4 + 2 * p] += wr * pr - wi * pi;
              acc[d][5 + 2 * p] += wr * pi + wi * pr;
            }
        }
      }
    }
#pragma unroll
    for (int d = 0; d < MAXD; ++d) {
      if (d >= D) break;
#pragma unroll
      for (int q = 0; q < REC; ++q) {
        float v = acc[d][q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == q) mx[(i * D + d) * REC + q] = v;
      }
    }
  }
}

// Polarisation-resolved bank: row records of Eq. hh_ieo grouped by
// delta = m_a - m_c (one warp per bank row), REC_P floats per detector:
//   [0..2]  delta = 0:  X0 = sum_a <h_a+|h_a+>, Y0 = sum_a 2 Re <h_a+|h_ax>, W0 = sum_a <h_ax|h_ax>
//   [3 + 6 (delta - 1) ...]  delta = 1..3, complex (re, im):
//           X = sum <h_a+|h_c+>, Y = sum (<h_a+|h_cx> + <h_ax|h_c+>), W = sum <h_ax|h_cx>  (a > c)
// with <h_j|h_j'>_d = sum_b omega_{d b} h_j h_j'^*, or, with relative binning
// (App. A, Eqs. hh_weights, h_h), sum_b W^{<h|h>}_{d j j' b} h_j h_j'^* over the
// (mode, polarisation) components j = 2m + p (RB: rb_hh [D][2M][2M][B]);
// master rows [Re h+ | Im h+ | Re hx | Im hx | 0].
template <bool RB>
__global__ void cross_terms_pol_kernel(int64_t n_rows, int64_t row0, int64_t I_bank, int M, int D, int B, int Kpad,
                                       int4 mode_m, const float *__restrict__ master,
                                       const float *__restrict__ omega, const double2 *__restrict__ rb_hh,
                                       float *__restrict__ mx) {
  extern __shared__ float om_s[];
  if (!RB) {
    for (int k = threadIdx.x; k < D * B; k += blockDim.x) om_s[k] = omega[k];
    __syncthreads();
  }
  const int mm[MAXM] = {mode_m.x, mode_m.y, mode_m.z, mode_m.w};
  const int J = 2 * M;
  const int lane = threadIdx.x & 31;
  const int64_t warp_global = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp_global; i < n_rows; i += nwarps) {
    float acc[MAXD][21];
#pragma unroll
    for (int d = 0; d < MAXD; ++d)
#pragma unroll
      for (int q = 0; q < 21; ++q) acc[d][q] = 0.f;
    for (int b = lane; b < B; b += 32) {
      float hr[MAXM][2], hi[MAXM][2];
#pragma unroll
      for (int m = 0; m < MAXM; ++m)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          if (m < M) {
            const float *row = master + ((int64_t)m * I_bank + row0 + i) * Kpad + 2 * q * B;
            hr[m][q] = __ldg(row + b);
            hi[m][q] = __ldg(row + B + b);
          } else {
            hr[m][q] = 0.f; hi[m][q] = 0.f;
          }
        }
#pragma unroll
      for (int d = 0; d < MAXD; ++d) {
        if (d >= D) break;
        const float om = RB ? 0.f : om_s[d * B + b];
        // weight of the component pair (j, j') at this bin, and w h_j h_j'^*
        auto wgt = [&](int j, int jp) -> float2 {
          if (!RB) return make_float2(om, 0.f);
          const double2 v = __ldg(&rb_hh[(((int64_t)d * J + j) * J + jp) * B + b]);
          return make_float2((float)v.x, (float)v.y);
        };
        auto term = [&](int a, int p, int c, int pc) -> float2 {
          const float pr = hr[a][p] * hr[c][pc] + hi[a][p] * hi[c][pc];
          const float pi = hi[a][p] * hr[c][pc] - hr[a][p] * hi[c][pc];
          const float2 w = wgt(2 * a + p, 2 * c + pc);
          return make_float2(w.x * pr - w.y * pi, w.x * pi + w.y * pr);
        };
#pragma unroll
        for (int a = 0; a < MAXM; ++a) {
          if (a >= M) break;
          acc[d][0] += term(a, 0, a, 0).x;
          acc[d][1] += 2.f * term(a, 0, a, 1).x;
          acc[d][2] += term(a, 1, a, 1).x;
        }
#pragma unroll
        for (int a = 1; a < MAXM; ++a)
#pragma unroll
          for (int c = 0; c < a; ++c) {
            if (a >= M) continue;
            const int g = 3 + 6 * (mm[a] - mm[c] - 1);
            // h_a+ h_c+^*, h_a+ h_cx^* + h_ax h_c+^*, h_ax h_cx^* (each with its weight)
            const float2 x = term(a, 0, c, 0), y1 = term(a, 0, c, 1), y2 = term(a, 1, c, 0), w = term(a, 1, c, 1);
#pragma unroll
            for (int z = 0; z < 3; ++z)
              if (g == 3 + 6 * z) {
                acc[d][3 + 6 * z] += x.x;
                acc[d][4 + 6 * z] += x.y;
                acc[d][5 + 6 * z] += y1.x + y2.x;
                acc[d][6 + 6 * z] += y1.y + y2.y;
                acc[d][7 + 6 * z] += w.x;
                acc[d][8 + 6 * z] += w.y;
              }
          }
      }
    }
#pragma unroll
    for (int d = 0; d < MAXD; ++d) {
      if (d >= D) break;
#pragma unroll
      for (int q = 0; q < 21; ++q) {
        float v = acc[d][q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == q) mx[(i * D + d) * REC_P + q] = v;
      }
      if (lane >= 21 && lane < REC_P) mx[(i * D + d) * REC_P + lane] = 0.f;
    }
  }
}

// ---------------------------------------------------------------------------
// Bank conversion (load time)
// ---------------------------------------------------------------------------
// complex [rows][M][B] (double2 or float2) -> FP32 master [M][I_bank][Kpad] rows [re | im]
template <typename CT>
__global__ void bank_to_master_kernel(int64_t rows, int64_t row0, int64_t I_bank, int M, int B, int Kpad, int NP,
                                      const CT *__restrict__ src, float *__restrict__ master,
                                      float *__restrict__ amax, int *status) {
  // src [rows][M][NP][B] -> master row (m, i): [Re h_0 | Im h_0 | Re h_1 | Im h_1 | pad]
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= rows * M * NP * B) return;
  int b = (int)(k % B);
  int64_t rq = k / B;
  int q = (int)(rq % NP);
  int64_t rm = rq / NP;
  int m = (int)(rm % M);
  int64_t r = rm / M;
  CT v = src[k];
  float re = (float)v.x, im = (float)v.y;
  if (!isfinite(re) || !isfinite(im)) { atomicCAS(status, 0, DEV_E_NONFINITE); re = 0.f; im = 0.f; }
  float *row = master + ((int64_t)m * I_bank + row0 + r) * Kpad + 2 * q * B;
  row[b] = re;
  row[B + b] = im;
  atomic_max_nonneg(amax, fmaxf(fabsf(re), fabsf(im)));
}
template __global__ void bank_to_master_kernel<double2>(int64_t, int64_t, int64_t, int, int, int, int,
                                                        const double2 *, float *, float *, int *);
template __global__ void bank_to_master_kernel<float2>(int64_t, int64_t, int64_t, int, int, int, int,
                                                       const float2 *, float *, float *, int *);

__global__ void master_to_planes_kernel(int64_t n, const float *__restrict__ master, const float *__restrict__ amax,
                                        __nv_bfloat16 *__restrict__ bf /*[2][n]*/, __half *__restrict__ hf /*[2][n]*/,
                                        float *__restrict__ scale_out) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  float sc = pow2_scale(*amax);
  if (k == 0) *scale_out = sc;
  if (k >= n) return;
  float v = master[k] * sc;
  __nv_bfloat16 hi = __float2bfloat16_rn(v);
  bf[k] = hi;
  bf[n + k] = __float2bfloat16_rn(v - __bfloat162float(hi));
  const float vh = v * FP16_OPERAND_SCALE;
  __half h = __float2half_rn(vh);
  hf[k] = h;
  hf[n + k] = __float2half_rn(vh - __half2float(h));
}

// ---------------------------------------------------------------------------
// K9: distance-marginal table (FP64)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double mu_d(double y) {
  double r = sqrt(y * y + 4.0);
  return y >= 0.0 ? 0.5 * (y + r) : 2.0 / (r - y);
}

// K(y, sigma) = ln E[(s+t)^-4] + 4 ln(s + mu(y)), t ~ N(y,1) truncated at 0, s = e^sigma.
__device__ double dm_K_exact(double y, double sig) {
  // 8-point Gauss-Legendre on composite panels (published nodes/weights)
  const double gx[4] = {0.1834346424956498, 0.5255324099163290, 0.7966664774136267, 0.9602898564975363};
  const double gw[4] = {0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};
  const double s = exp(sig);
  // weight w(t) = exp(-(t-y)^2/2 + c) with c = y^2/2 for y < 0 (no underflow near t = 0)
  const bool neg = y < 0.0;
  const double T = neg ? fmin(40.0, 40.0 / fmax(-y, 1.0)) + 1.0 : y + 9.0;
  const double wneg = neg ? 1.0 / fmax(-y, 1.0) : 1e30;
  double num = 0.0, t = 0.0;
  int guard = 0;
  while (t < T && guard < 4000) {
    double hwid = fmin(0.5, 0.5 * (s + t));
    hwid = fmin(hwid, wneg);
    hwid = fmin(hwid, T - t);
    double cen = t + 0.5 * hwid, hl = 0.5 * hwid, acc = 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      for (int sg = -1; sg <= 1; sg += 2) {
        double tt = cen + sg * hl * gx[j];
        double lw = neg ? (-0.5 * tt * tt + tt * y) : (-0.5 * (tt - y) * (tt - y));
        double g = s + tt;
        double g2 = g * g;
        acc += gw[j] * exp(lw) / (g2 * g2);
      }
    }
    num += acc * hl;
    t += hwid;
    ++guard;
  }
  const double SQ2PI = 2.5066282746310002;
  double den = neg ? SQ2PI * 0.5 * erfcx(-y * 0.70710678118654752) : SQ2PI * (1.0 - 0.5 * erfc(y * 0.70710678118654752));
  return log(num / den) + 4.0 * log(s + mu_d(y));
}

__global__ void build_dm_table_kernel(float4 *__restrict__ tab) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= DM_NY * DM_NS) return;
  int iy = k % DM_NY, is = k / DM_NY;
  double y = dm_node_y(iy);
  double sg = (double)DM_S0 + (double)DM_DS * is;
  const double h = 1e-3;
  double f = dm_K_exact(y, sg);
  double fyp = dm_K_exact(y + h, sg), fym = dm_K_exact(y - h, sg);
  double fsp = dm_K_exact(y, sg + h), fsm = dm_K_exact(y, sg - h);
  double fpp = dm_K_exact(y + h, sg + h), fpm = dm_K_exact(y + h, sg - h);
  double fmp = dm_K_exact(y - h, sg + h), fmm = dm_K_exact(y - h, sg - h);
  double fy = (fyp - fym) / (2 * h), fs = (fsp - fsm) / (2 * h);
  double fys = (fpp - fpm - fmp + fmm) / (4 * h * h);
  // y-derivatives unscaled (cells have different widths), sigma-derivatives times ds
  tab[k] = make_float4((float)f, (float)fy, (float)(fs * DM_DS), (float)(fys * DM_DS));
}

__global__ void dist_marg_eval_kernel(int64_t n, const float *__restrict__ dh, const float *__restrict__ hh,
                                      float u_min, const float4 *__restrict__ tab, float *__restrict__ out) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < n) out[k] = dm_lnlbar(dh[k], hh[k], u_min, tab);
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static inline unsigned nblk(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

void launch_prep(const PrepArgs &a, cudaStream_t st) {
  const bool pol = (a.n_pol == 2);
  const int NP = pol ? 2 : 1;
  // data weights per (mode, polarisation) component: c [D][M NP][B]
  prep_bins_kernel<<<nblk((int64_t)a.D * a.B, 256), 256, 0, st>>>(a.D, a.B, a.M * NP, a.f, a.w, a.psd, a.data,
                                                                a.rb_dh, a.c, a.omega, a.fh, a.fl, a.status);
  if (a.sqrt_dd) {
    if (a.rb_dh) rb_norm_kernel<<<1, 256, 0, st>>>(a.D, a.M * NP, a.B, a.rb_dh, a.rb_hh, a.sqrt_dd);
    else data_norm_kernel<<<1, 256, 0, st>>>(a.D, a.B, a.w, a.psd, a.data, a.sqrt_dd);
  }
  prep_ext_kernel<<<nblk(a.E * a.D, 256), 256, 0, st>>>(a.E, a.D, a.M, a.t, a.R, pol ? a.F : nullptr, a.th, a.tl,
                                                        a.Rf, a.qx, a.status);
  if (pol)
    build_G_pol_kernel<<<nblk(a.E * a.B, 256), 256, 0, st>>>(a.E, a.D, a.M, a.B, a.fh, a.fl, a.th, a.tl, a.c, a.F,
                                                             a.G32, a.gmax);
  else
    build_G_kernel<<<nblk(a.E * a.B, 256), 256, 0, st>>>(a.E, a.D, a.M, a.B, a.fh, a.fl, a.th, a.tl, a.c, a.Rf,
                                                         a.G32, a.gmax);
  const int pad = a.Kpad - 2 * NP * a.B;
  const int64_t n = (int64_t)a.M * a.E * (a.B > pad ? a.B : pad);
  if (a.pack_kind == 0)
    pack_G_kernel<float><<<nblk(n, 256), 256, 0, st>>>(a.E, a.M, a.B, a.Kpad, NP, a.G32, a.gmax, 0, 1, a.gpack,
                                                       a.gscale);
  else if (a.pack_kind == 1)
    pack_G_kernel<__nv_bfloat16><<<nblk(n, 256), 256, 0, st>>>(a.E, a.M, a.B, a.Kpad, NP, a.G32, a.gmax, 1,
                                                               a.pack_planes, a.gpack, a.gscale);
  else
    pack_G_kernel<__half><<<nblk(n, 256), 256, 0, st>>>(a.E, a.M, a.B, a.Kpad, NP, a.G32, a.gmax, 2, a.pack_planes,
                                                        a.gpack, a.gscale);
}

// ---------------------------------------------------------------------------
// Pre-selection operand (Sec. IV.D, App. B): G_k[b, t] = c_{kb} e^{-2 pi i f_b t_{kt}}
// ---------------------------------------------------------------------------
// One matrix for every mode (plain quadrature), or one per mode when the data
// weights are per mode (relative binning): G[mg][(d, t)][b], mg < n_gmodes.
__global__ void presel_G_kernel(int D, int B, int M, int n_gmodes, int n_t, int n_tpad, const float *__restrict__ fh,
                                const float *__restrict__ fl, const double *__restrict__ t_grid,
                                const float2 *__restrict__ c, float2 *__restrict__ G, float *__restrict__ gmax,
                                int *status) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  float a = 0.f;
  if (k < (int64_t)n_gmodes * D * n_tpad * B) {
    const int b = (int)(k % B);
    const int64_t mcol = k / B;
    const int col = (int)(mcol % ((int64_t)D * n_tpad));
    const int mg = (int)(mcol / ((int64_t)D * n_tpad));
    const int d = col / n_tpad, t = col - d * n_tpad;
    float2 g = make_float2(0.f, 0.f);
    if (t < n_t) {
      double tv = t_grid[(int64_t)d * n_t + t];
      if (!isfinite(tv)) { atomicCAS(status, 0, DEV_E_NONFINITE); tv = 0.0; }
      const float th = (float)tv, tl = (float)(tv - (double)th);
      const float2 T = shift_factor(fh[b], fl[b], th, tl);
      const float2 cc = c[((int64_t)d * M + mg) * B + b];
      g = make_float2(T.x * cc.x - T.y * cc.y, T.x * cc.y + T.y * cc.x);
    }
    G[k] = g;
    a = fmaxf(fabsf(g.x), fabsf(g.y));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(gmax, a);
}

void launch_presel_prep(const PreselPrepArgs &a, cudaStream_t st) {
  const int DB = a.D * a.B;
  prep_bins_kernel<<<nblk(DB > a.B ? DB : a.B, 256), 256, 0, st>>>(a.D, a.B, a.M, a.f, a.w, a.psd, a.data,
                                                                   a.rb_dh, a.c, a.omega, a.fh, a.fl, a.status);
  const int mg = a.rb_dh ? a.M : 1;
  const int64_t n = (int64_t)mg * a.D * a.n_tpad * a.B;
  presel_G_kernel<<<nblk(n, 256), 256, 0, st>>>(a.D, a.B, a.M, mg, a.n_t, a.n_tpad, a.fh, a.fl, a.t_grid, a.c,
                                                a.G32, a.gmax, a.status);
  if (a.pack_kind == 0) return;  // the FP32 operand is used as it is
  const int64_t E = (int64_t)a.D * a.n_tpad;
  const int pad = a.Kpad - 2 * a.B;
  const int64_t np = mg * E * (a.B > pad ? a.B : pad);
  if (a.pack_kind == 1)
    pack_G_kernel<__nv_bfloat16><<<nblk(np, 256), 256, 0, st>>>(E, mg, a.B, a.Kpad, 1, a.G32, a.gmax, 1, a.pack_planes,
                                                                a.gpack, a.gscale);
  else
    pack_G_kernel<__half><<<nblk(np, 256), 256, 0, st>>>(E, mg, a.B, a.Kpad, 1, a.G32, a.gmax, 2, a.pack_planes,
                                                         a.gpack, a.gscale);
}

// GT[mat][b][t] = G[mat][t][b]: one thread per output element, t fastest, so
// the writes are coalesced (the operand is a few MB: the strided reads stay in L2).
__global__ void transpose_G_kernel(int64_t n_mat, int T, int B, const float2 *__restrict__ G,
                                   float2 *__restrict__ GT) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n_mat * B * T) return;
  const int t = (int)(k % T);
  const int64_t mb = k / T;
  const int b = (int)(mb % B);
  const int64_t mat = mb / B;
  GT[k] = G[(mat * T + t) * B + b];
}

void launch_transpose_G(int64_t n_mat, int T, int B, const float2 *G, float2 *GT, cudaStream_t st) {
  transpose_G_kernel<<<nblk(n_mat * B * T, 256), 256, 0, st>>>(n_mat, T, B, G, GT);
}

// Gp[q][2c + p][b] = G32[c][b] if q == p, else 0: the polarisation-resolved
// pre-selection's operand rows before packing (one row per (column, polarisation)).
__global__ void presel_pol_spread_kernel(int64_t n_cols, int B, const float2 *__restrict__ G32,
                                         float2 *__restrict__ Gp) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= 4 * n_cols * B) return;
  const int b = (int)(k % B);
  const int64_t r = k / B;                    // q * 2 n_cols + 2c + p
  const int64_t e = r % (2 * n_cols), q = r / (2 * n_cols);
  const int64_t c = e >> 1, p = e & 1;
  Gp[k] = (q == p) ? G32[c * B + b] : make_float2(0.f, 0.f);
}

void launch_presel_pol_pack(int64_t n_cols, int B, int Kpad, const float2 *G32, float2 *Gp, const float *gmax,
                            int kind, int planes, void *out, float *scale_out, cudaStream_t st) {
  presel_pol_spread_kernel<<<nblk(4 * n_cols * B, 256), 256, 0, st>>>(n_cols, B, G32, Gp);
  const int64_t E = 2 * n_cols;
  const int pad = Kpad - 4 * B;
  const int64_t n = E * (B > pad ? B : pad);
  if (kind == 1)
    pack_G_kernel<__nv_bfloat16><<<nblk(n, 256), 256, 0, st>>>(E, 1, B, Kpad, 2, Gp, gmax, 1, planes, out,
                                                               scale_out);
  else
    pack_G_kernel<__half><<<nblk(n, 256), 256, 0, st>>>(E, 1, B, Kpad, 2, Gp, gmax, 2, planes, out, scale_out);
}

void launch_cross_terms(int64_t n_rows, int64_t row0, int64_t I_bank, int M, int D, int B, int Kpad,
                        const float *master, const float *omega, const double2 *rb_hh, float *mx, int n_sms,
                        cudaStream_t st) {
  int bs = 256;
  int64_t warps = (n_rows + 0);
  int64_t blocks = (warps * 32 + bs - 1) / bs;
  int64_t cap = (int64_t)n_sms * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  if (rb_hh) {
    cross_terms_kernel<true><<<(unsigned)blocks, bs, 0, st>>>(n_rows, row0, I_bank, M, D, B, Kpad, master, omega,
                                                              rb_hh, mx);
    return;
  }
  // omega [D][B] staged in shared memory (the caller keeps D B floats within 227 KB)
  size_t smem = sizeof(float) * (size_t)D * B;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(cross_terms_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cross_terms_kernel<false><<<(unsigned)blocks, bs, smem, st>>>(n_rows, row0, I_bank, M, D, B, Kpad, master, omega,
                                                                nullptr, mx);
}

void launch_bank_to_master(int64_t rows, int64_t row0, int64_t I_bank, int M, int B, int Kpad, int NP,
                           const void *src, int dtype, float *master, float *amax, int *status, cudaStream_t st) {
  int64_t n = rows * M * NP * B;
  if (dtype == DOTPE_C128)
    bank_to_master_kernel<double2><<<nblk(n, 256), 256, 0, st>>>(rows, row0, I_bank, M, B, Kpad, NP,
                                                                 (const double2 *)src, master, amax, status);
  else
    bank_to_master_kernel<float2><<<nblk(n, 256), 256, 0, st>>>(rows, row0, I_bank, M, B, Kpad, NP,
                                                                (const float2 *)src, master, amax, status);
}

void launch_cross_terms_pol(int64_t n_rows, int64_t row0, int64_t I_bank, int M, int D, int B, int Kpad,
                            const int *mode_m, const float *master, const float *omega, const double2 *rb_hh,
                            float *mx, int n_sms, cudaStream_t st) {
  int bs = 256;
  int64_t blocks = (n_rows * 32 + bs - 1) / bs;
  int64_t cap = (int64_t)n_sms * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  const int4 mm = make_int4(mode_m[0], M > 1 ? mode_m[1] : 0, M > 2 ? mode_m[2] : 0, M > 3 ? mode_m[3] : 0);
  if (rb_hh) {
    cross_terms_pol_kernel<true><<<(unsigned)blocks, bs, 0, st>>>(n_rows, row0, I_bank, M, D, B, Kpad, mm, master,
                                                                  omega, rb_hh, mx);
    return;
  }
  const size_t smem = sizeof(float) * (size_t)D * B;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(cross_terms_pol_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cross_terms_pol_kernel<false><<<(unsigned)blocks, bs, smem, st>>>(n_rows, row0, I_bank, M, D, B, Kpad, mm, master,
                                                                    omega, nullptr, mx);
}

// dst[o][r][w] = src[o][rows[r]][w] (32-bit words): a bank's rows gathered into a new bank
__global__ void gather_rows_kernel(int64_t outer, int64_t src_rows, int64_t n, int64_t row_words,
                                   const uint32_t *__restrict__ src, const int64_t *__restrict__ rows,
                                   uint32_t *__restrict__ dst) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= outer * n * row_words) return;
  const int64_t w = k % row_words, orr = k / row_words;
  const int64_t r = orr % n, o = orr / n;
  dst[k] = src[(o * src_rows + rows[r]) * row_words + w];
}

void launch_gather_rows(int64_t outer, int64_t src_rows, int64_t n, int64_t row_words, const void *src,
                        const int64_t *rows, void *dst, cudaStream_t st) {
  gather_rows_kernel<<<nblk(outer * n * row_words, 256), 256, 0, st>>>(outer, src_rows, n, row_words,
                                                                      (const uint32_t *)src, rows, (uint32_t *)dst);
}

void launch_master_to_planes(int64_t n, const float *master, const float *amax, __nv_bfloat16 *bf, __half *hf,
                             float *scale_out, cudaStream_t st) {
  master_to_planes_kernel<<<nblk(n, 256), 256, 0, st>>>(n, master, amax, bf, hf, scale_out);
}

// The distance-marginal table is a constant of the method, the same for every
// context: it lives in this static device array (3.2 MB, held by every GPU
// that loads the library until the process exits) and is built once per CUDA
// context of a device, by the first dotpe context created there, instead of
// once per dotpe context.
static __device__ __align__(256) float4 g_dm_table[DM_NY * DM_NS];

static unsigned long long current_ctx_id();

int shared_dm_table(int device, cudaStream_t st, float4 **tab, char *msg, size_t msg_len) {
  static std::mutex mu;
  static float4 *addr[64] = {nullptr};
  static unsigned long long addr_ctx[64] = {0};
  if (device < 0 || device >= 64) {
    snprintf(msg, msg_len, "device %d out of range", device);
    return DOTPE_E_INVALID;
  }
  std::lock_guard<std::mutex> lk(mu);
  // the caller has made `device` current
  const unsigned long long cid = current_ctx_id();
  if (!addr[device] || cid == 0 || cid != addr_ctx[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_dm_table);
    if (e == cudaSuccess && p == nullptr) e = cudaErrorInvalidSymbol;
    if (e == cudaSuccess) {
      build_dm_table_kernel<<<nblk((int64_t)DM_NY * DM_NS, 64), 64, 0, st>>>((float4 *)p);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      snprintf(msg, msg_len, "table build: %s", cudaGetErrorString(e));
      return DOTPE_E_DEVICE;
    }
    addr[device] = (float4 *)p;
    addr_ctx[device] = cid;
  }
  *tab = addr[device];
  return DOTPE_OK;
}

void launch_dist_marg_eval(int64_t n, const float *dh, const float *hh, float u_min, const float4 *tab, float *out,
                           cudaStream_t st) {
  dist_marg_eval_kernel<<<nblk(n, 256), 256, 0, st>>>(n, dh, hh, u_min, tab, out);
}


// ---------------------------------------------------------------------------
// Allocation-free distance-marginal evaluation.
//
// Scratch for the inputs and the output lives in this file-scope device array
// (3 x DM_NOALLOC_MAX floats = 12 MiB), which every GPU that loads the library
// holds until the process exits.  Host code cannot use the array's name as a
// device address (on the host it is only a stand-in), so its address is looked
// up once per device with cudaGetSymbolAddress and cached.  Every call shares
// the one array: calls that overlap on the GPU (from different streams or
// threads without ordering) race on it.  Each call overwrites exactly the
// entries it reads before reading them, so nothing has to start at zero.
// ---------------------------------------------------------------------------
static __device__ __align__(256) float g_dm_noalloc_scratch[3 * DM_NOALLOC_MAX];

// Identity of the current CUDA context (0 if the driver cannot tell): the
// scratch array's address belongs to a context, so a device reset, which tears
// the primary context down, must lead to a fresh look-up.
static unsigned long long current_ctx_id() {
  typedef CUresult (*GetCurrent)(CUcontext *);
  typedef CUresult (*GetId)(CUcontext, unsigned long long *);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *f1 = nullptr, *f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess)
      get_current = (GetCurrent)f1;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q2 == cudaDriverEntryPointSuccess)
      get_id = (GetId)f2;
  }
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (get_current && get_id && get_current(&c) == CUDA_SUCCESS && c && get_id(c, &id) == CUDA_SUCCESS) return id;
  return 0;
}

int dist_marg_eval_noalloc(int device, int64_t n, const float *dh, const float *hh, float u_min, const float4 *tab,
                           float *out, cudaStream_t st, char *msg, size_t msg_len) {
  static std::mutex mu;
  static float *addr[64] = {nullptr};
  static unsigned long long addr_ctx[64] = {0};
  if (n < 0 || n > DM_NOALLOC_MAX) {
    snprintf(msg, msg_len, "n=%lld exceeds the allocation-free limit of %lld evaluations per call", (long long)n,
             (long long)DM_NOALLOC_MAX);
    return DOTPE_E_INVALID;
  }
  if (device < 0 || device >= 64) {
    snprintf(msg, msg_len, "device %d out of range", device);
    return DOTPE_E_INVALID;
  }
  if (n == 0) return DOTPE_OK;
  float *base = nullptr;
  {
    std::lock_guard<std::mutex> lk(mu);
    // the caller has made `device` current; its context has been set up by the runtime
    const unsigned long long cid = current_ctx_id();
    if (!addr[device] || cid == 0 || cid != addr_ctx[device]) {
      // first use on this device (or in a new context of it)
      void *p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_dm_noalloc_scratch);
      if (e != cudaSuccess || p == nullptr) {
        snprintf(msg, msg_len, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        return DOTPE_E_DEVICE;
      }
      addr[device] = (float *)p;
      addr_ctx[device] = cid;
    }
    base = addr[device];
  }
  float *s_dh = base, *s_hh = base + DM_NOALLOC_MAX, *s_out = base + 2 * DM_NOALLOC_MAX;
  cudaError_t e = cudaMemcpyAsync(s_dh, dh, (size_t)n * 4, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s_hh, hh, (size_t)n * 4, cudaMemcpyDefault, st);
  if (e == cudaSuccess) {
    dist_marg_eval_kernel<<<nblk(n, 256), 256, 0, st>>>(n, s_dh, s_hh, u_min, tab, s_out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, s_out, (size_t)n * 4, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    snprintf(msg, msg_len, "%s", cudaGetErrorString(e));
    return DOTPE_E_DEVICE;
  }
  return DOTPE_OK;
}

}  // namespace dotpe
