// Pre-selection kernels' host side and the finish kernels; the tensor-core
// kernel is in kernel_presel.cuh, instantiated here for the shared time-grid
// operand (VAR 0) and in kernel_presel_permode.cu / kernel_presel_polres.cu for the
// per-mode (relative binning) and polarisation-resolved operands, so that the
// three instantiation sets compile in parallel.
#include "kernel_presel.cuh"

namespace dotpe {

template <int VAR>
cudaError_t launch_presel_var(const CUtensorMap &mapG, const CUtensorMap &mapBank, const PreselParams &p, bool bf16,
                              bool split, int grid, cudaStream_t st);
template <>
cudaError_t launch_presel_var<0>(const CUtensorMap &mapG, const CUtensorMap &mapBank, const PreselParams &p,
                                 bool bf16, bool split, int grid, cudaStream_t st) {
  return launch_presel_pm<0>(mapG, mapBank, p, bf16, split, grid, st);
}

// Per row: ln L^ML_{ik} and (o, t) from the packed maxima, ln L^inco.ML_i =
// sum_k (FP64), and the running maximum of ln L^inco.ML (order-preserving
// bits of a non-negative double).
__global__ void presel_rows_kernel(int64_t n, int D, int n_phi, const unsigned long long *__restrict__ keys,
                                   float *__restrict__ ml, int *__restrict__ arg_ot, double *__restrict__ inco,
                                   unsigned long long *max_bits) {
  __shared__ unsigned long long smax[8];
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  unsigned long long mb = 0;
  if (i < n) {
    double s = 0.0;
    for (int k = 0; k < D; ++k) {
      const unsigned long long key = keys[i * D + k];
      const float v = __uint_as_float((uint32_t)(key >> 32));
      const uint32_t idx = 0xffffffffu - (uint32_t)(key & 0xffffffffu);
      ml[i * D + k] = v;
      arg_ot[(i * D + k) * 2] = (int)(idx % (uint32_t)n_phi);
      arg_ot[(i * D + k) * 2 + 1] = (int)(idx / (uint32_t)n_phi);
      s += (double)v;
    }
    inco[i] = s;
    mb = (unsigned long long)__double_as_longlong(s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, mb, o);
    mb = v > mb ? v : mb;
  }
  if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = mb;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long m = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) m = smax[q] > m ? smax[q] : m;
    atomicMax(max_bits, m);
  }
}

// Sec. IV.D selection: rows with ln L^inco.ML >= max - delta, in increasing
// order, and the lowest row that attains the maximum.  One block of 1024
// threads; each round covers 8192 rows (8 consecutive per thread).
__global__ void presel_select_kernel(int64_t n, double delta, const double *__restrict__ inco,
                                     const unsigned long long *max_bits, int64_t *__restrict__ sel,
                                     PreselOut *out) {
  __shared__ long long wsum[32];
  __shared__ long long s_arg;
  const double mx = __longlong_as_double((long long)*max_bits);
  const double thr = mx - delta;
  if (threadIdx.x == 0) s_arg = n;
  __syncthreads();
  long long pos = 0;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t base = 0; base < n; base += 8 * 1024) {
    const int64_t r0 = base + (int64_t)threadIdx.x * 8;
    int cnt = 0;
    int64_t first_max = n;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int64_t r = r0 + q;
      if (r < n) {
        const double v = inco[r];
        cnt += v >= thr;
        if (v == mx && r < first_max) first_max = r;
      }
    }
    if (first_max < n) atomicMin(&s_arg, (long long)first_max);
    // block-wide exclusive scan of cnt
    long long x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
      long long v = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
      }
      wsum[lane] = v;  // inclusive over warps
    }
    __syncthreads();
    long long at = pos + (wid > 0 ? wsum[wid - 1] : 0) + x - cnt;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int64_t r = r0 + q;
      if (r < n && inco[r] >= thr) sel[at++] = r;
    }
    pos += wsum[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out->max_inco = mx;
    out->threshold = thr;
    out->arg_i = s_arg < n ? s_arg : 0;
    out->n_selected = pos;
  }
}

int launch_presel(const CUtensorMap &mapG, const CUtensorMap &mapBank, const PreselParams &p, bool bf16, bool split,
                  bool per_mode, bool pol, int n_sms, cudaStream_t st) {
  const int total = p.n_itile * p.n_ctile;
  const int grid = total < n_sms ? (total > 0 ? total : 1) : n_sms;
  const cudaError_t e = pol ? launch_presel_var<2>(mapG, mapBank, p, bf16, split, grid, st)
                            : per_mode ? launch_presel_var<1>(mapG, mapBank, p, bf16, split, grid, st)
                                       : launch_presel_var<0>(mapG, mapBank, p, bf16, split, grid, st);
  return (int)e;
}

void launch_presel_finish(int64_t n, int D, int n_phi, double delta, const unsigned long long *keys, float *ml,
                          int *arg_ot, double *inco, unsigned long long *max_bits, int64_t *sel, PreselOut *out,
                          cudaStream_t st) {
  const int64_t blocks = (n + 255) / 256;
  presel_rows_kernel<<<(unsigned)(blocks > 0 ? blocks : 1), 256, 0, st>>>(n, D, n_phi, keys, ml, arg_ot, inco,
                                                                          max_bits);
  presel_select_kernel<<<1, 1024, 0, st>>>(n, delta, inco, max_bits, sel, out);
}

}  // namespace dotpe
