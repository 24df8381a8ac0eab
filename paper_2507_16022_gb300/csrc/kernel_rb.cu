// Relative-binning weights (App. A, Eqs. dh_weights, hh_weights).
//
// The components m are the bank's modes, or its (mode, polarisation) pairs
// m = 2 m_az + p for a polarisation-resolved bank (W_{kmpb}, W_{kmm'pp'b}); up to
// 2 MAXM of them.  For detector d, component m (and m') and coarse node b:
//   W^{<d|h>}_{d m b}    = sum_n 4 dff_n d_d(f_n) h0_dm^*(f_n) s_b(f_n) / S_d(f_n)  /  h0_dm^*(f_b)
//   W^{<h|h>}_{d m m' b} = sum_n 4 dff_n h0_dm(f_n) h0_dm'^*(f_n) s_b(f_n) / S_d(f_n) / (h0_dm(f_b) h0_dm'^*(f_b))
// with h0_dm(f) = h0_m(f) e^{-2 pi i f t0_d} (the reference arriving at the
// detector at t0_d) and s_b the piecewise-linear hat function of node b on the
// fine grid (1 at f_b, 0 at the neighbouring nodes), so the sums run over the
// fine points between nodes b-1 and b+1.  One block per (d, b), FP64
// accumulation (the weights are made once per event), a fixed-order block
// reduction.  W^{<h|h>} is Hermitian in (m, m'): the upper triangle is summed
// and mirrored.
#include "common.cuh"
#include "kernels.h"

namespace dotpe {

namespace {
constexpr int RB_THREADS = 256;
// NC: components per weight set, MAXM modes or 2 MAXM (mode, polarisation) pairs
template <int NC> struct RbAcc {
  static constexpr int NPAIR = NC * (NC + 1) / 2;  // upper triangle m <= m'
  static constexpr int NACC = 2 * (NC + NPAIR);    // re, im of the dh and hh sums
};

// e^{-2 pi i f t} in FP64 (the phase reduced with sincospi of the product f t)
__device__ __forceinline__ double2 shift64(double f, double t) {
  double s, c;
  sincospi(2.0 * f * t, &s, &c);
  return make_double2(c, -s);
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // a b^*
  return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double den = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}
}  // namespace

template <int NC>
__global__ void __launch_bounds__(RB_THREADS)
    rb_weights_kernel(int D, int M, int64_t N, const double *__restrict__ ff, const double *__restrict__ dff,
                      const double *__restrict__ psd, const double2 *__restrict__ data,
                      const double2 *__restrict__ h0, const double *__restrict__ t0, int B,
                      const int64_t *__restrict__ node, double2 *__restrict__ w_dh, double2 *__restrict__ w_hh,
                      int *status) {
  constexpr int RB_NACC = RbAcc<NC>::NACC;
  __shared__ double red[RB_THREADS / 32][RB_NACC];
  __shared__ double fn3[3];
  const int d = blockIdx.x / B, b = blockIdx.x % B;
  if (d >= D) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // the node frequencies this block's hat function needs (fn3 = f_{b-1}, f_b, f_{b+1})
  if (tid < 3) {
    const int bb = b - 1 + tid;
    fn3[tid] = (bb >= 0 && bb < B) ? ff[node[bb]] : 0.0;
  }
  __syncthreads();
  const double fbm = fn3[0], fb = fn3[1], fbp = fn3[2];
  const int64_t n0 = node[b > 0 ? b - 1 : 0], n1 = node[b < B - 1 ? b + 1 : B - 1];
  const double td = t0 ? t0[d] : 0.0;
  double acc[RB_NACC];
#pragma unroll
  for (int q = 0; q < RB_NACC; ++q) acc[q] = 0.0;
  for (int64_t n = n0 + tid; n <= n1; n += RB_THREADS) {
    const double f = ff[n];
    double s;
    if (b > 0 && f >= fbm && f <= fb) s = (f - fbm) / (fb - fbm);
    else if (b < B - 1 && f >= fb && f <= fbp) s = (fbp - f) / (fbp - fb);
    else s = (f == fb) ? 1.0 : 0.0;
    if (s == 0.0) continue;
    const double S = psd[(int64_t)d * N + n];
    const double wgt = 4.0 * dff[n] * s / S;
    if (!(S > 0.0) || !isfinite(wgt)) {
      atomicCAS(status, 0, DEV_E_NONFINITE);
      continue;
    }
    const double2 T = shift64(f, td);
    const double2 dd = data[(int64_t)d * N + n];
    double2 hv[NC];
#pragma unroll
    for (int m = 0; m < NC; ++m) hv[m] = (m < M) ? cmul(h0[(int64_t)m * N + n], T) : make_double2(0.0, 0.0);
#pragma unroll
    for (int m = 0; m < NC; ++m) {
      const double2 v = cmulc(dd, hv[m]);  // d h0^*
      acc[2 * m] += wgt * v.x;
      acc[2 * m + 1] += wgt * v.y;
    }
    int p = 0;
#pragma unroll
    for (int m = 0; m < NC; ++m)
#pragma unroll
      for (int mp = m; mp < NC; ++mp, ++p) {
        const double2 v = cmulc(hv[m], hv[mp]);  // h0_m h0_m'^*
        acc[2 * NC + 2 * p] += wgt * v.x;
        acc[2 * NC + 2 * p + 1] += wgt * v.y;
      }
  }
  // block reduction (fixed order: warp shuffles, then warp 0 over the warps)
#pragma unroll
  for (int q = 0; q < RB_NACC; ++q) {
    double v = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][q] = v;
  }
  __syncthreads();
  if (tid == 0) {
    double tot[RB_NACC];
    for (int q = 0; q < RB_NACC; ++q) {
      double v = 0.0;
      for (int w = 0; w < RB_THREADS / 32; ++w) v += red[w][q];
      tot[q] = v;
    }
    const double2 T = shift64(fb, td);
    double2 hb[NC];
    for (int m = 0; m < NC; ++m) {
      hb[m] = (m < M) ? cmul(h0[(int64_t)m * N + node[b]], T) : make_double2(1.0, 0.0);
      if (m < M && hb[m].x == 0.0 && hb[m].y == 0.0) atomicCAS(status, 0, DEV_E_SHAPE);
    }
    for (int m = 0; m < M; ++m) {
      const double2 num = make_double2(tot[2 * m], tot[2 * m + 1]);
      w_dh[((int64_t)d * M + m) * B + b] = cdiv(num, make_double2(hb[m].x, -hb[m].y));
    }
    int p = 0;
    for (int m = 0; m < NC; ++m)
      for (int mp = m; mp < NC; ++mp, ++p) {
        if (m >= M || mp >= M) continue;
        const double2 num = make_double2(tot[2 * NC + 2 * p], tot[2 * NC + 2 * p + 1]);
        const double2 w = cdiv(num, cmulc(hb[m], hb[mp]));
        w_hh[(((int64_t)d * M + m) * M + mp) * B + b] = w;
        if (mp != m) w_hh[(((int64_t)d * M + mp) * M + m) * B + b] = make_double2(w.x, -w.y);
      }
  }
}

void launch_rb_weights(int D, int M, int64_t N, const double *ff, const double *dff, const double *psd,
                       const double2 *data, const double2 *h0, const double *t0, int B, const int64_t *node,
                       double2 *w_dh, double2 *w_hh, int *status, cudaStream_t st) {
  if (M <= MAXM)
    rb_weights_kernel<MAXM><<<(unsigned)(D * B), RB_THREADS, 0, st>>>(D, M, N, ff, dff, psd, data, h0, t0, B, node,
                                                                      w_dh, w_hh, status);
  else
    rb_weights_kernel<2 * MAXM><<<(unsigned)(D * B), RB_THREADS, 0, st>>>(D, M, N, ff, dff, psd, data, h0, t0, B,
                                                                          node, w_dh, w_hh, status);
}

}  // namespace dotpe
