// K6: cross-tile reduction in FP64 (Eq. Z_sum with w_o = 1; Eqs. posterior_element,
// int_ess, ext_ess).  Each fused-kernel tile left log-sum-exp partials (max, sum) in
// FP32; they are combined here in double precision.
//   ln S1 = ln sum_ieo p_ieo,  ln S2 = ln sum_ieo p_ieo^2,  p_ieo = w_i w_e Lbar_ieo
//   ln Z  = ln S1 - ln(N_i N_e N_phi)
//   N_eff = S1^2 / S2, N_eff,int = S1^2 / sum_i P_i^2, N_eff,ext = S1^2 / sum_e P_e^2
#include "common.cuh"
#include "kernels.h"

namespace dotpe {

struct DLse {
  double m, s;
  __device__ void init() { m = -INFINITY; s = 0.0; }
  __device__ void add_ms(double om, double os) {
    if (om == -INFINITY || !(os > 0.0)) return;
    if (m == -INFINITY) { m = om; s = os; return; }
    if (om > m) { s = s * exp(m - om) + os; m = om; }
    else s += os * exp(om - m);
  }
  __device__ double value() const { return (m == -INFINITY) ? -INFINITY : m + log(s); }
};

// ln P_i over the e-tiles (row partials [n_etile][n_int])
__global__ void reduce_rows_kernel(int64_t n, int nparts, const float2 *__restrict__ part, double *__restrict__ out) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  DLse a;
  a.init();
  for (int p = 0; p < nparts; ++p) {
    float2 v = part[(int64_t)p * n + k];
    a.add_ms((double)v.x, (double)v.y);
  }
  out[k] = a.value();
}

__device__ void block_lse(DLse &a, double *sm, double *ss) {
  const int t = threadIdx.x;
  sm[t] = a.m;
  ss[t] = a.s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (t < w) {
      DLse x;
      x.m = sm[t];
      x.s = ss[t];
      x.add_ms(sm[t + w], ss[t + w]);
      sm[t] = x.m;
      ss[t] = x.s;
    }
    __syncthreads();
  }
  a.m = sm[0];
  a.s = ss[0];
  __syncthreads();
}

__global__ void __launch_bounds__(1024) reduce_final_kernel(ReduceArgs a) {
  __shared__ double sm[1024], ss[1024];
  __shared__ float bml[1024];
  __shared__ long long barg[1024];
  __shared__ long long bnp[1024];
  const int t = threadIdx.x, nt = blockDim.x;
  const int64_t n_tiles = (int64_t)a.n_itile * a.n_etile;
  DLse s1, s2, ri, ce;
  s1.init(); s2.init(); ri.init(); ce.init();
  float best = -1.f;
  long long arg = 0x7fffffffffffffffLL, np = 0;
  for (int64_t k = t; k < n_tiles; k += nt) {
    float4 v = a.tile_part[k];
    s1.add_ms(v.x, v.y);
    s2.add_ms(v.z, v.w);
    float ml = a.tile_ml[k];
    long long g = a.tile_arg[k];
    if (ml > best || (ml == best && g < arg)) { best = ml; arg = g; }
    np += a.tile_npass[k];
  }
  for (int64_t k = t; k < a.n_int; k += nt) {
    double v = a.ln_p_int[k];
    if (v != -INFINITY) ri.add_ms(2.0 * v, 1.0);
  }
  for (int64_t k = t; k < a.n_ext; k += nt) {
    double v = a.ln_p_ext[k];
    if (v != -INFINITY) ce.add_ms(2.0 * v, 1.0);
  }
  block_lse(s1, sm, ss);
  block_lse(s2, sm, ss);
  block_lse(ri, sm, ss);
  block_lse(ce, sm, ss);
  bml[t] = best;
  barg[t] = arg;
  bnp[t] = np;
  __syncthreads();
  for (int w = nt / 2; w > 0; w >>= 1) {
    if (t < w) {
      if (bml[t + w] > bml[t] || (bml[t + w] == bml[t] && barg[t + w] < barg[t])) {
        bml[t] = bml[t + w];
        barg[t] = barg[t + w];
      }
      bnp[t] += bnp[t + w];
    }
    __syncthreads();
  }
  if (t == 0) {
    ReduceOut o;
    double l1 = s1.value(), l2 = s2.value();
    o.ln_s1 = l1;
    o.ln_s2 = l2;
    o.ln_z = l1 - log((double)a.n_int) - log((double)a.n_ext) - log((double)a.n_phi);
    o.n_eff = (l1 == -INFINITY) ? 0.0 : exp(2.0 * l1 - l2);
    o.n_eff_int = (l1 == -INFINITY) ? 0.0 : exp(2.0 * l1 - ri.value());
    o.n_eff_ext = (l1 == -INFINITY) ? 0.0 : exp(2.0 * l1 - ce.value());
    o.max_ml = bml[0];
    o.arg = barg[0];
    o.n_marg = bnp[0];
    o.threshold = (a.cut_delta > 0.f) ? (double)(*a.ml_running) - (double)a.cut_delta : -INFINITY;
    o.status = *a.status;
    o.pad = 0;
    *a.out = o;
  }
}

void launch_reduce(const ReduceArgs &a, cudaStream_t st) {
  reduce_rows_kernel<<<(unsigned)((a.n_int + 255) / 256), 256, 0, st>>>(a.n_int, a.n_etile, a.row_part, a.ln_p_int);
  reduce_rows_kernel<<<(unsigned)((a.n_ext + 255) / 256), 256, 0, st>>>(a.n_ext, a.n_itile, a.col_part, a.ln_p_ext);
  reduce_final_kernel<<<1, 1024, 0, st>>>(a);
}

}  // namespace dotpe
