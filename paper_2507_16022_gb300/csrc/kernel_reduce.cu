// K6: cross-tile reduction (Eq. Z_sum with w_o = 1; Eqs. posterior_element,
// int_ess, ext_ess).  Each fused-kernel tile left log-sum-exp partials (max, sum)
// in FP32; they are combined with FP64 accumulation:
//   ln S1 = ln sum_ieo p_ieo,  ln S2 = ln sum_ieo p_ieo^2,  p_ieo = w_i w_e Lbar_ieo
//   ln Z  = ln S1 - ln(N_i N_e N_phi)
//   N_eff = S1^2 / S2, N_eff,int = S1^2 / sum_i P_i^2, N_eff,ext = S1^2 / sum_e P_e^2
// Two passes per log-sum-exp: the maximum (FP32, exact), then the sum of
// s * exp(m - max) with the exponential and the accumulation in FP64, so that
// the combination adds only FP64 rounding to the FP32 partials.
// A slice processed as several bank blocks merges each block's (max, sum) pairs,
// its column marginals and its best ln L^ML into FP64 accumulators in block
// order; the final kernel turns them into the evidence.
#include "common.cuh"
#include "kernels.h"

namespace dotpe {

namespace {
constexpr int RB = 256;  // threads per block
constexpr int NB = 128;  // blocks of the parallel passes
constexpr int NQ = 3;    // log-sum-exp inputs of a bank block: tile m1, tile m2, 2 ln P_i
}

// ln P over partials [nparts][n] (row or column marginal).  A block takes 32
// consecutive entries (coalesced) and splits the parts over its 8 thread rows;
// each thread keeps an online (max, sum) in FP64 and the rows merge in shared
// memory.  With acc != nullptr the value is merged into the FP64 accumulator
// acc[k] = (m, s) (s = 0: empty) instead of written to out.
constexpr int LX = 32, LY = 8;

__device__ __forceinline__ void lse_add(double &m, double &s, double x, double w) {
  if (!(w > 0.0)) return;
  if (!(s > 0.0)) { m = x; s = w; return; }
  if (x > m) { s = s * exp(m - x) + w; m = x; }
  else s += w * exp(x - m);
}
// The same for FP32 partials: FP32 maximum and exponentials (the partials carry
// FP32 precision), FP64 sum.
__device__ __forceinline__ void lse_add_f(float &m, double &s, float x, float w) {
  if (!(w > 0.f)) return;
  if (!(s > 0.0)) { m = x; s = w; return; }
  if (x > m) { s = s * (double)__expf(m - x) + (double)w; m = x; }
  else s += (double)w * (double)__expf(x - m);
}

__global__ void __launch_bounds__(LX * LY) reduce_lines_kernel(int64_t n, int nparts, const float2 *__restrict__ part,
                                                               double *__restrict__ out, double2 *__restrict__ acc,
                                                               int first) {
  __shared__ double sm[LY][LX], ss[LY][LX];
  const int64_t k = blockIdx.x * (int64_t)LX + threadIdx.x;
  float mf = 0.f;
  double s = 0.0;
  if (k < n)
    for (int p = threadIdx.y; p < nparts; p += LY) {
      const float2 v = part[(int64_t)p * n + k];
      lse_add_f(mf, s, v.x, v.y);
    }
  double m = mf;
  sm[threadIdx.y][threadIdx.x] = m;
  ss[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y != 0 || k >= n) return;
  for (int y = 1; y < LY; ++y) lse_add(m, s, sm[y][threadIdx.x], ss[y][threadIdx.x]);
  if (!acc) {
    out[k] = (s > 0.0) ? m + log(s) : -INFINITY;
    return;
  }
  double2 a = first ? make_double2(0.0, 0.0) : acc[k];
  lse_add(a.x, a.y, m, s);
  acc[k] = a;
}

__device__ __forceinline__ float block_max(float v, float *sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = (threadIdx.x < blockDim.x / 32) ? sh[threadIdx.x] : -INFINITY;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) sh[0] = v;
  }
  __syncthreads();
  v = sh[0];
  __syncthreads();
  return v;
}

__device__ __forceinline__ double block_sum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = (threadIdx.x < blockDim.x / 32) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) sh[0] = v;
  }
  __syncthreads();
  v = sh[0];
  __syncthreads();
  return v;
}

// Pass 1 over one bank block: per-block maxima of the log-sum-exp inputs, the
// argmax and the marginalised count.
__global__ void __launch_bounds__(RB) reduce_pass1_kernel(ReduceArgs a, float *__restrict__ bmax,
                                                           float *__restrict__ bml, long long *__restrict__ barg,
                                                           long long *__restrict__ bnp) {
  __shared__ float shf[32];
  __shared__ double shd[32];
  __shared__ float sv[RB];
  __shared__ long long sa[RB];
  const int64_t n_tiles = (int64_t)a.n_itile * a.n_etile;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t k0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  float m1 = -INFINITY, m2 = -INFINITY, mr = -INFINITY, best = -1.f;
  long long arg = 0x7fffffffffffffffLL, np = 0;
  for (int64_t k = k0; k < n_tiles; k += stride) {
    float4 v = a.tile_part[k];
    if (v.y > 0.f) m1 = fmaxf(m1, v.x);
    if (v.w > 0.f) m2 = fmaxf(m2, v.z);
    float ml = a.tile_ml[k];
    long long g = a.tile_arg[k];
    if (ml > best || (ml == best && g < arg)) { best = ml; arg = g; }
    np += a.tile_npass[k];
  }
  const double *lpi = a.ln_p_int + a.row_offset;
  for (int64_t k = k0; k < a.n_int; k += stride) mr = fmaxf(mr, (float)(2.0 * lpi[k]));
  float r[NQ] = {m1, m2, mr};
  for (int q = 0; q < NQ; ++q) {
    float v = block_max(r[q], shf);
    if (threadIdx.x == 0) bmax[q * gridDim.x + blockIdx.x] = v;
  }
  sv[threadIdx.x] = best;
  sa[threadIdx.x] = arg;
  __syncthreads();
  for (int w = RB / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      if (sv[threadIdx.x + w] > sv[threadIdx.x] ||
          (sv[threadIdx.x + w] == sv[threadIdx.x] && sa[threadIdx.x + w] < sa[threadIdx.x])) {
        sv[threadIdx.x] = sv[threadIdx.x + w];
        sa[threadIdx.x] = sa[threadIdx.x + w];
      }
    }
    __syncthreads();
  }
  double npd = block_sum((double)np, shd);  // counts < 2^53
  if (threadIdx.x == 0) {
    bml[blockIdx.x] = sv[0];
    barg[blockIdx.x] = sa[0];
    bnp[blockIdx.x] = (long long)npd;
  }
}

// Pass 2: per-block FP64 sums of s * exp(m - M) against the bank block's maxima.
__global__ void __launch_bounds__(RB) reduce_pass2_kernel(ReduceArgs a, const float *__restrict__ bmax,
                                                           double *__restrict__ bsum) {
  __shared__ double shd[32];
  __shared__ float M[NQ];
  if (threadIdx.x < NQ) {
    float m = -INFINITY;
    for (int b = 0; b < (int)gridDim.x; ++b) m = fmaxf(m, bmax[threadIdx.x * gridDim.x + b]);
    M[threadIdx.x] = m;
  }
  __syncthreads();
  const int64_t n_tiles = (int64_t)a.n_itile * a.n_etile;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t k0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double s[NQ] = {0.0, 0.0, 0.0};
  for (int64_t k = k0; k < n_tiles; k += stride) {
    float4 v = a.tile_part[k];
    if (v.y > 0.f) s[0] += (double)v.y * exp((double)v.x - (double)M[0]);
    if (v.w > 0.f) s[1] += (double)v.w * exp((double)v.z - (double)M[1]);
  }
  const double *lpi = a.ln_p_int + a.row_offset;
  for (int64_t k = k0; k < a.n_int; k += stride) {
    double v = lpi[k];
    if (v != -INFINITY) s[2] += exp(2.0 * v - (double)M[2]);
  }
  for (int q = 0; q < NQ; ++q) {
    double v = block_sum(s[q], shd);
    if (threadIdx.x == 0) bsum[q * gridDim.x + blockIdx.x] = v;
  }
}

__device__ __forceinline__ void acc_merge(double &am, double &as, double bm, double bs) {
  if (!(bs > 0.0)) return;
  if (!(as > 0.0)) { am = bm; as = bs; return; }
  if (bm > am) { as = as * exp(am - bm) + bs; am = bm; }
  else as += bs * exp(bm - am);
}

// Merges one bank block into the event's FP64 accumulators (fixed order: deterministic).
__global__ void reduce_block_merge_kernel(ReduceArgs a, int nb, const float *__restrict__ bmax,
                                          const double *__restrict__ bsum, const float *__restrict__ bml,
                                          const long long *__restrict__ barg, const long long *__restrict__ bnp) {
  // one warp; lane l takes the per-block entries l, l + 32, ...; fixed shuffle order
  const int lane = threadIdx.x;
  double m[NQ], sm[NQ];
  for (int q = 0; q < NQ; ++q) {
    float mq = -INFINITY;
    double sq = 0.0;
    for (int b = lane; b < nb; b += 32) {
      mq = fmaxf(mq, bmax[q * nb + b]);
      sq += bsum[q * nb + b];
    }
    for (int o = 16; o > 0; o >>= 1) {
      mq = fmaxf(mq, __shfl_xor_sync(0xffffffffu, mq, o));
      sq += __shfl_xor_sync(0xffffffffu, sq, o);
    }
    m[q] = mq;
    sm[q] = sq;
  }
  // arguments are packed ((i * n_ext + e) * n_phi + o) with i relative to the block
  const long long shift = (long long)a.row_offset * a.n_ext * a.n_phi;
  float best = -1.f;
  long long arg = 0x7fffffffffffffffLL, np = 0;
  for (int b = lane; b < nb; b += 32) {
    const long long g = barg[b] + shift;
    if (bml[b] > best || (bml[b] == best && g < arg)) { best = bml[b]; arg = g; }
    np += bnp[b];
  }
  for (int o = 16; o > 0; o >>= 1) {
    const float ob = __shfl_xor_sync(0xffffffffu, best, o);
    const long long oa = __shfl_xor_sync(0xffffffffu, arg, o);
    if (ob > best || (ob == best && oa < arg)) { best = ob; arg = oa; }
    np += __shfl_xor_sync(0xffffffffu, np, o);
  }
  if (lane != 0) return;
  EvAcc c = a.first ? EvAcc{0.0, 0.0, 0.0, 0.0, 0.0, 0.0, -1.f, 0x7fffffffffffffffLL, 0} : *a.acc;
  double *dst[NQ][2] = {{&c.s1_m, &c.s1_s}, {&c.s2_m, &c.s2_s}, {&c.pi_m, &c.pi_s}};
  for (int q = 0; q < NQ; ++q)
    if (m[q] != -INFINITY) acc_merge(*dst[q][0], *dst[q][1], m[q], sm[q]);
  if (best > c.best || (best == c.best && arg < c.arg)) { c.best = best; c.arg = arg; }
  c.n_marg += np;
  *a.acc = c;
}

// After the last block: column marginals, Sum_e P_e^2 (two passes) and the evidence.
__global__ void __launch_bounds__(1024) reduce_final_kernel(ReduceArgs a) {
  __shared__ float shf[32];
  __shared__ double shd[32];
  const EvAcc c = *a.acc;
  float mc = -INFINITY;
  for (int64_t k = threadIdx.x; k < a.n_ext; k += blockDim.x) {
    const double2 v = a.acc_col[k];
    const double l = (v.y > 0.0) ? v.x + log(v.y) : -INFINITY;
    a.ln_p_ext[k] = l;
    mc = fmaxf(mc, (float)(2.0 * l));
  }
  mc = block_max(mc, shf);
  double sc = 0.0;
  if (mc != -INFINITY)
    for (int64_t k = threadIdx.x; k < a.n_ext; k += blockDim.x) {
      const double l = a.ln_p_ext[k];
      if (l != -INFINITY) sc += exp(2.0 * l - (double)mc);
    }
  sc = block_sum(sc, shd);
  if (threadIdx.x != 0) return;
  auto lnv = [](double m, double s) { return (s > 0.0) ? m + log(s) : -INFINITY; };
  const double l1 = lnv(c.s1_m, c.s1_s), l2 = lnv(c.s2_m, c.s2_s), lpi = lnv(c.pi_m, c.pi_s);
  const double lpe = (mc == -INFINITY || !(sc > 0.0)) ? -INFINITY : (double)mc + log(sc);
  ReduceOut o;
  o.ln_s1 = l1;
  o.ln_s2 = l2;
  o.ln_z = l1 - log((double)a.n_int_total) - log((double)a.n_ext) - log((double)a.n_phi);
  o.n_eff = (l1 == -INFINITY) ? 0.0 : exp(2.0 * l1 - l2);
  o.n_eff_int = (l1 == -INFINITY) ? 0.0 : exp(2.0 * l1 - lpi);
  o.n_eff_ext = (l1 == -INFINITY) ? 0.0 : exp(2.0 * l1 - lpe);
  o.max_ml = c.best;
  o.arg = c.arg;
  o.n_marg = c.n_marg;
  o.threshold = (a.cut_delta > 0.f) ? (double)(*a.ml_running) - (double)a.cut_delta : -INFINITY;
  o.status = *a.status;
  o.n_refined = a.n_refined ? *a.n_refined : -1;
  o.n_cand = a.n_cand ? (long long)a.n_cand[0] : -1;
  o.n_eval = a.n_cand ? (long long)a.n_cand[1] : -1;
  *a.out = o;
}

size_t reduce_scratch_bytes() {
  return (size_t)NB * (NQ * sizeof(float) + NQ * sizeof(double) + sizeof(float) + 2 * sizeof(long long)) + 256;
}

void launch_reduce_block(const ReduceArgs &a, cudaStream_t st) {
  const dim3 lb(LX, LY);
  reduce_lines_kernel<<<(unsigned)((a.n_int + LX - 1) / LX), lb, 0, st>>>(a.n_int, a.n_etile, a.row_part,
                                                                         a.ln_p_int + a.row_offset, nullptr, 0);
  reduce_lines_kernel<<<(unsigned)((a.n_ext + LX - 1) / LX), lb, 0, st>>>(a.n_ext, a.n_itile, a.col_part, nullptr,
                                                                         a.acc_col, a.first);
  uint8_t *w = (uint8_t *)a.scratch;
  float *bmax = (float *)w;
  double *bsum = (double *)(w + NB * NQ * sizeof(float));
  float *bml = (float *)(bsum + NB * NQ);
  long long *barg = (long long *)(((uintptr_t)(bml + NB) + 7) & ~(uintptr_t)7);
  long long *bnp = barg + NB;
  reduce_pass1_kernel<<<NB, RB, 0, st>>>(a, bmax, bml, barg, bnp);
  reduce_pass2_kernel<<<NB, RB, 0, st>>>(a, bmax, bsum);
  reduce_block_merge_kernel<<<1, 32, 0, st>>>(a, NB, bmax, bsum, bml, barg, bnp);
}

void launch_reduce_final(const ReduceArgs &a, cudaStream_t st) { reduce_final_kernel<<<1, 1024, 0, st>>>(a); }

// ---------------------------------------------------------------------------
// Refinement selection (after a screening pass).  Tile t of event k is refined
// when its screened best ln L^ML reaches max_k - window - 2 margin(max_k): the
// exact value of any pair differs from its screened one by at most one margin,
// and so does the exact maximum.  Two kernels keep the list in event order and
// banded tile order within an event: per-block counts, then each block writes
// its items at the prefix of the earlier counts.
// ---------------------------------------------------------------------------
namespace {
constexpr int SB = 1024;  // tiles per selection block
}

__device__ __forceinline__ bool select_tile(const SelectBatch &a, int w, int &k, int &t) {
  if (w >= a.begin[a.n]) return false;
  int lo = 0, hi = a.n - 1;  // largest k with begin[k] <= w
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.begin[mid] <= w) lo = mid;
    else hi = mid - 1;
  }
  k = lo;
  const SelectEvent &v = a.ev[k];
  int it, et;
  super_tile(w - a.begin[k], v.n_itile, v.n_etile, v.band, it, et);
  t = it * v.n_etile + et;
  const float mx = *v.ml_screen;
  const float thr = mx - v.window - 2.f * screen_margin(mx, v.margin_k, *v.sqrt_dd);
  return v.tile_ml[t] >= thr;
}

__global__ void __launch_bounds__(SB) select_count_kernel(SelectBatch a) {
  int k = -1, t;
  const bool f = select_tile(a, blockIdx.x * SB + threadIdx.x, k, t);
  const int c = __syncthreads_count(f);
  if (threadIdx.x == 0) a.counts[blockIdx.x] = c;
  // per-event counts: one atomic per (warp, event)
  const unsigned grp = __match_any_sync(0xffffffffu, f ? k : -1);
  const int lane = threadIdx.x & 31;
  if (f && lane == __ffs(grp) - 1) atomicAdd(a.ev[k].n_refined, __popc(grp));
}

__global__ void __launch_bounds__(SB) select_write_kernel(SelectBatch a) {
  __shared__ int wsum[SB / 32];
  __shared__ int base_s;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // prefix of the earlier blocks' counts (and, in block 0, the total)
  {
    const int upto = (blockIdx.x == 0) ? (int)gridDim.x : (int)blockIdx.x;
    int v = 0;
    for (int q = tid; q < upto; q += SB) v += a.counts[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) wsum[wid] = v;
    __syncthreads();
    if (tid == 0) {
      int s = 0;
      for (int q = 0; q < SB / 32; ++q) s += wsum[q];
      base_s = (blockIdx.x == 0) ? 0 : s;
      if (blockIdx.x == 0) *a.n_list = s;
    }
    __syncthreads();
  }
  int k = 0, t = 0;
  const bool f = select_tile(a, blockIdx.x * SB + tid, k, t);
  const unsigned bal = __ballot_sync(0xffffffffu, f);
  if (lane == 0) wsum[wid] = __popc(bal);
  __syncthreads();
  if (tid == 0) {
    int s = 0;
    for (int q = 0; q < SB / 32; ++q) {
      const int c = wsum[q];
      wsum[q] = s;
      s += c;
    }
  }
  __syncthreads();
  if (f) a.list[base_s + wsum[wid] + __popc(bal & ((1u << lane) - 1u))] = make_int2(k, t);
}

// Per event: the frozen refinement maximum; the refined-tile count starts at 0.
__global__ void select_events_kernel(SelectBatch a) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.n) return;
  const SelectEvent &v = a.ev[k];
  const float mx = *v.ml_screen;
  *v.ml_refine = fmaxf(mx - screen_margin(mx, v.margin_k, *v.sqrt_dd), 0.f);
  *v.n_refined = 0;
  if (a.sep) a.sep[k] = (mx > v.sep_ml) ? 1 : 0;
}

int select_count_blocks(int n_tiles) { return (n_tiles + SB - 1) / SB; }

void launch_select(const SelectBatch &a, cudaStream_t st) {
  const int nb = select_count_blocks(a.begin[a.n]);
  if (nb < 1) return;
  select_events_kernel<<<(a.n + 63) / 64, 64, 0, st>>>(a);
  select_count_kernel<<<nb, SB, 0, st>>>(a);
  select_write_kernel<<<nb, SB, 0, st>>>(a);
}

}  // namespace dotpe
