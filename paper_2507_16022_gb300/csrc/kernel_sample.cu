// Posterior samples of a finished event: resampling with the weights
// p_ieo = w_i w_e w_o Lbar_ieo (Eq. posterior_element; Sec. III resampling;
// w_o = 1) and a distance per sample drawn from the summand of the distance
// marginal (App. C: phase and distance drawn per (intrinsic, extrinsic) pair).
//
// Per sample, four uniforms in [0, 1):
//   u1 -> i  from the row marginals ln sum_{e,o} p_ieo (the event's FP64 row weights),
//   u2 -> e  from row i of the stored ln Lbar_ie plus ln w_e,
//   u3 -> o  from the pair's phases that pass the event's ML cut, weights Lbar_ieo
//            (the pair recomputed in FP64 from the event's inputs: per-mode
//            components and mode overlaps, Eqs. dh_ieo, hh_ieo, per (mode,
//            polarisation) component with real antenna patterns F_edp for a
//            polarisation-resolved bank; Lbar from the same device distance
//            marginal as the fused kernels),
//   u4 -> d_L / d_L^0 = 1/u from the density of u on [u_min, inf),
//            proportional to u^-4 exp(dh u - hh u^2 / 2) (pi(d_L) ~ d_L^2).
// Each draw takes the smallest index whose cumulative weight exceeds u times
// the total.  The distance is inverted on a 1,024-node grid of v = sqrt(hh) u
// over [s, max(s, x, v*) + 12] (x = dh/sqrt(hh), s = sqrt(hh) u_min), the
// log-density linear within each interval (integrated and inverted in closed
// form).  One warp per sample.
#include "common.cuh"
#include "dist_marg.cuh"
#include "kernels.h"

namespace dotpe {

namespace {
constexpr int SW = 8;         // samples (warps) per block
constexpr int SNODE = 1024;   // distance grid nodes
constexpr int SPL = SNODE / 32;

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double wmax(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
// inclusive prefix sum over the warp's lanes
__device__ __forceinline__ double wscan(double v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  return v;
}

// The warp draws an index from weights exp(x_k - xmax), k in [0, n), held in
// contiguous chunks per lane (get(k) evaluates x_k): the smallest k whose
// cumulative weight exceeds u * total.  Returns -1 if the total is zero.
template <typename Get>
__device__ int warp_pick(int n, double u, int lane, Get get) {
  const int chunk = (n + 31) / 32;
  const int k0 = min(n, lane * chunk), k1 = min(n, k0 + chunk);
  double mx = -INFINITY;
  for (int k = k0; k < k1; ++k) mx = fmax(mx, get(k));
  mx = wmax(mx);
  if (!(mx > -INFINITY)) return -1;
  double loc = 0.0;
  for (int k = k0; k < k1; ++k) loc += exp(get(k) - mx);
  const double incl = wscan(loc, lane);
  const double total = __shfl_sync(0xffffffffu, incl, 31);
  const double target = u * total;
  const double excl = incl - loc;
  int pick = -1;
  if (excl <= target && target < incl) {
    double c = excl;
    for (int k = k0; k < k1; ++k) {
      c += exp(get(k) - mx);
      if (c > target) { pick = k; break; }
    }
    if (pick < 0) pick = k1 - 1;
  }
  const unsigned has = __ballot_sync(0xffffffffu, pick >= 0);
  if (!has) {  // target at the very top (rounding): the last index of positive weight
    int last = -1;
    for (int k = k0; k < k1; ++k)
      if (get(k) > -INFINITY) last = k;
    const unsigned hl = __ballot_sync(0xffffffffu, last >= 0);
    return __shfl_sync(0xffffffffu, last, 31 - __clz(hl));
  }
  return __shfl_sync(0xffffffffu, pick, __ffs(has) - 1);
}
}  // namespace

// Cumulative row weights: cdf[i] = sum_{i' <= i} exp(ln_p[i'] - max), one block.
__global__ void sample_row_cdf_kernel(int64_t n, const double *__restrict__ ln_p, double *__restrict__ cdf) {
  __shared__ double red[1024 / 32];
  __shared__ double s_max;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t chunk = (n + blockDim.x - 1) / blockDim.x;
  const int64_t k0 = min(n, (int64_t)tid * chunk), k1 = min(n, k0 + chunk);
  double mx = -INFINITY;
  for (int64_t k = k0; k < k1; ++k) mx = fmax(mx, ln_p[k]);
  mx = wmax(mx);
  if (lane == 0) red[w] = mx;
  __syncthreads();
  if (tid == 0) {
    double m = -INFINITY;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) m = fmax(m, red[q]);
    s_max = m;
  }
  __syncthreads();
  const double M = s_max;
  double loc = 0.0;
  for (int64_t k = k0; k < k1; ++k) loc += (M > -INFINITY) ? exp(ln_p[k] - M) : 0.0;
  // exclusive scan of the chunk sums over the block
  double incl = wscan(loc, lane);
  __syncthreads();
  if (lane == 31) red[w] = incl;
  __syncthreads();
  if (w == 0) {
    double v = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
    v = wscan(v, lane);
    red[lane] = v;
  }
  __syncthreads();
  double c = (w > 0 ? red[w - 1] : 0.0) + incl - loc;
  for (int64_t k = k0; k < k1; ++k) {
    c += (M > -INFINITY) ? exp(ln_p[k] - M) : 0.0;
    cdf[k] = c;
  }
}

// NP = 2: polarisation-resolved bank, components j = (m, p) with master row
// [Re h_m+ | Im h_m+ | Re h_mx | Im h_mx] and response F_edp (real).
template <int NP>
__global__ void __launch_bounds__(SW * 32)
    sample_kernel(const SampleArgs a, int64_t n, const double *__restrict__ uni, const double *__restrict__ cdf,
                  int64_t *__restrict__ i_out, int64_t *__restrict__ e_out, int32_t *__restrict__ o_out,
                  double *__restrict__ d_out) {
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int64_t s = blockIdx.x * (int64_t)SW + wl;
  if (s >= n) return;  // warp-uniform
  const double u1 = uni[4 * s], u2 = uni[4 * s + 1], u3 = uni[4 * s + 2], u4 = uni[4 * s + 3];
  const int M = a.n_modes, D = a.n_det, B = a.n_bins;
  // ---- i: the smallest row whose cumulative weight exceeds u1 * total
  int64_t i = 0;
  if (lane == 0) {
    const double target = u1 * cdf[a.n_int - 1];
    int64_t lo = 0, hi = a.n_int - 1;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (cdf[mid] > target) hi = mid;
      else lo = mid + 1;
    }
    i = lo;
  }
  i = __shfl_sync(0xffffffffu, i, 0);
  // ---- e: row i of the stored ln Lbar_ie plus ln w_e
  const float *row = a.lnl + i * a.n_ext;
  const int e = warp_pick((int)a.n_ext, u2, lane, [&](int k) {
    const float v = row[k];
    return (v == -INFINITY) ? -INFINITY : (double)v + (a.lw_ext ? a.lw_ext[k] : 0.0);
  });
  // ---- the pair in FP64, per component j = (m, p): z_j = sum_d R_edj sum_b c_dmb T_db h_j(b),
  // H_jj' = sum_d R_edj R_edj'^* sum_b W h_j h_j'^* (R_edj = R_edm, or F_edp for NP = 2)
  constexpr int MJ = MAXM * NP;
  const int J = M * NP;
  double zr[MJ] = {}, zi[MJ] = {};
  double Hr[MJ][MJ] = {}, Hi[MJ][MJ] = {};
  const int64_t ib = a.i_base + i;
  for (int d = 0; d < D; ++d) {
    double Sr[MJ] = {}, Si[MJ] = {};
    double Qr[MJ][MJ] = {}, Qi[MJ][MJ] = {};
    const double td = (e >= 0) ? a.t[(int64_t)e * D + d] : 0.0;
    for (int b = lane; b < B; b += 32) {
      double s_, c_;
      sincospi(2.0 * a.f[b] * td, &s_, &c_);
      const double Tr = c_, Ti = -s_;
      double hr[MJ], hi[MJ];
#pragma unroll
      for (int j = 0; j < MJ; ++j) {
        const int m = j / NP, p = j % NP;
        const float *row = a.master + ((int64_t)m * a.bank_rows + ib) * a.kpad + 2 * p * B;
        hr[j] = (j < J) ? (double)row[b] : 0.0;
        hi[j] = (j < J) ? (double)row[B + b] : 0.0;
      }
#pragma unroll
      for (int j = 0; j < MJ; ++j) {
        if (j >= J) break;
        const int m = j / NP;
        double cr, ci;
        if (a.rb_dh) {
          const double2 w = a.rb_dh[((int64_t)d * J + j) * B + b];
          cr = w.x; ci = -w.y;
        } else {
          const double om = 4.0 * a.w[b] / a.psd[(int64_t)d * B + b];
          const double2 dd = a.data[(int64_t)d * B + b];
          cr = om * dd.x; ci = -om * dd.y;
        }
        // (c T) h_j
        const double ctr = cr * Tr - ci * Ti, cti = cr * Ti + ci * Tr;
        Sr[j] += ctr * hr[j] - cti * hi[j];
        Si[j] += ctr * hi[j] + cti * hr[j];
#pragma unroll
        for (int jp = 0; jp < MJ; ++jp) {
          if (jp >= J) break;
          double wr, wi;
          if (a.rb_hh) {
            const double2 w = a.rb_hh[(((int64_t)d * J + j) * J + jp) * B + b];
            wr = w.x; wi = w.y;
          } else {
            wr = 4.0 * a.w[b] / a.psd[(int64_t)d * B + b]; wi = 0.0;
          }
          const double pr = hr[j] * hr[jp] + hi[j] * hi[jp], pi = hi[j] * hr[jp] - hr[j] * hi[jp];
          Qr[j][jp] += wr * pr - wi * pi;
          Qi[j][jp] += wr * pi + wi * pr;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < MJ; ++j) {
      Sr[j] = wsum(Sr[j]);
      Si[j] = wsum(Si[j]);
#pragma unroll
      for (int jp = 0; jp < MJ; ++jp) {
        Qr[j][jp] = wsum(Qr[j][jp]);
        Qi[j][jp] = wsum(Qi[j][jp]);
      }
    }
    if (e >= 0) {
      auto resp = [&](int j) -> double2 {
        if (NP == 2) return make_double2(a.F[((int64_t)e * D + d) * 2 + (j % 2)], 0.0);
        return a.R[((int64_t)e * D + d) * M + j];
      };
#pragma unroll
      for (int j = 0; j < MJ; ++j) {
        if (j >= J) break;
        const double2 R = resp(j);
        zr[j] += R.x * Sr[j] - R.y * Si[j];
        zi[j] += R.x * Si[j] + R.y * Sr[j];
#pragma unroll
        for (int jp = 0; jp < MJ; ++jp) {
          if (jp >= J) break;
          const double2 Rp = resp(jp);
          const double rr = R.x * Rp.x + R.y * Rp.y, ri = R.y * Rp.x - R.x * Rp.y;  // R R'^*
          Hr[j][jp] += rr * Qr[j][jp] - ri * Qi[j][jp];
          Hi[j][jp] += rr * Qi[j][jp] + ri * Qr[j][jp];
        }
      }
    }
  }
  // ---- o: phases that pass the cut, weights Lbar_ieo
  const int np = a.n_phi;
  auto dhh = [&](int o, double &dh, double &hh) {
    dh = 0.0;
    hh = 0.0;
#pragma unroll
    for (int j = 0; j < MJ; ++j) {
      if (j >= J) break;
      const int mj = a.mode_m[j / NP];
      const int km = (mj * o) % np;
      double sn, cs;
      sincospi(2.0 * (double)km / (double)np, &sn, &cs);
      dh += zr[j] * cs - zi[j] * sn;
#pragma unroll
      for (int jp = 0; jp < MJ; ++jp) {
        if (jp >= J) break;
        int kd = ((mj - a.mode_m[jp / NP]) * o) % np;
        if (kd < 0) kd += np;
        double s2, c2;
        sincospi(2.0 * (double)kd / (double)np, &s2, &c2);
        hh += Hr[j][jp] * c2 - Hi[j][jp] * s2;
      }
    }
  };
  const int o = (e < 0) ? -1 : warp_pick(np, u3, lane, [&](int k) {
    double dh, hh;
    dhh(k, dh, hh);
    const double ml = (dh > 0.0 && hh > 0.0) ? dh * dh / (2.0 * hh) : 0.0;
    if (!(ml >= a.threshold)) return (double)-INFINITY;
    return (double)dm_lnlbar((float)dh, (float)hh, a.u_min, a.dm_table);
  });
  // ---- distance
  double dist = 0.0;
  if (o >= 0) {
    double dh, hh;
    dhh(o, dh, hh);
    if (!(hh > 0.0)) {
      dist = cbrt(1.0 - u4) / (double)a.u_min;
    } else {
      const double r = sqrt(hh), x = dh / r, sv = r * (double)a.u_min;
      double vmax = sv;
      if (x > 4.0) vmax = fmax(vmax, 0.5 * (x + sqrt(x * x - 16.0)));
      const double vhi = fmax(fmax(sv, x), vmax) + 12.0;
      const double h = (vhi - sv) / (SNODE - 1);
      auto phi = [&](int k) {
        const double v = sv + k * h;
        return -4.0 * log(v) - 0.5 * (v - x) * (v - x);
      };
      // interval k = [v_k, v_{k+1}], k < SNODE - 1; lane holds intervals [lane SPL, lane SPL + SPL)
      double pm = -INFINITY;
      for (int q = 0; q < SPL; ++q) pm = fmax(pm, phi(lane * SPL + q));
      pm = wmax(pm);
      auto area = [&](int k) {
        if (k >= SNODE - 1) return 0.0;
        const double p0 = phi(k) - pm, p1 = phi(k + 1) - pm;
        const double dp = p1 - p0;
        return (fabs(dp) < 1e-12) ? h * exp(p0) : h * (exp(p1) - exp(p0)) / dp;
      };
      double loc = 0.0;
      for (int q = 0; q < SPL; ++q) loc += area(lane * SPL + q);
      const double incl = wscan(loc, lane);
      const double total = __shfl_sync(0xffffffffu, incl, 31);
      const double target = u4 * total;
      double vres = -1.0;
      if (incl - loc <= target && target < incl) {
        double c = incl - loc;
        for (int q = 0; q < SPL; ++q) {
          const int k = lane * SPL + q;
          const double ak = area(k);
          if (c + ak > target && k < SNODE - 1) {
            const double p0 = phi(k) - pm, p1 = phi(k + 1) - pm;
            const double sl = (p1 - p0) / h, rem = target - c;
            const double v0 = sv + k * h;
            vres = (fabs(sl) < 1e-12) ? v0 + rem / exp(p0) : v0 + log1p(sl * rem / exp(p0)) / sl;
            break;
          }
          c += ak;
        }
      }
      const unsigned has = __ballot_sync(0xffffffffu, vres >= 0.0);
      vres = has ? __shfl_sync(0xffffffffu, vres, __ffs(has) - 1) : vhi;
      dist = r / vres;
    }
  }
  if (lane == 0) {
    if (i_out) i_out[s] = i;
    if (e_out) e_out[s] = e;
    if (o_out) o_out[s] = o;
    if (d_out) d_out[s] = dist;
    if (e < 0 || o < 0) atomicCAS(a.status, 0, DEV_E_SHAPE);
  }
}

void launch_sample(const SampleArgs &a, int64_t n, const double *uni, double *cdf, int64_t *i_out, int64_t *e_out,
                   int32_t *o_out, double *d_out, cudaStream_t st) {
  sample_row_cdf_kernel<<<1, 1024, 0, st>>>(a.n_int, a.ln_p_int, cdf);
  const int64_t blocks = (n + SW - 1) / SW;
  if (a.n_pol == 2)
    sample_kernel<2><<<(unsigned)blocks, SW * 32, 0, st>>>(a, n, uni, cdf, i_out, e_out, o_out, d_out);
  else
    sample_kernel<1><<<(unsigned)blocks, SW * 32, 0, st>>>(a, n, uni, cdf, i_out, e_out, o_out, d_out);
}

}  // namespace dotpe
