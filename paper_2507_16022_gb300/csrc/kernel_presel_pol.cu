// Incoherent single-detector pre-selection (Sec. IV.D, App. B) of a
// polarisation-resolved bank, in FP32 on the CUDA cores.
//
// For bank row i, detector k, arrival time t_{kt} and phase phi_o:
//   Z_{ikmpt}     = sum_b h_{imp}(f_b) c_{kb} e^{-2 pi i f_b t_{kt}}       (Eq. dh_itop, per component)
//   <d|h>_{iktop} = Re sum_m e^{i m phi_o} Z_{ikmpt}
//   <h|h>_{ikopp'}: from the row's records of the bank's own overlaps grouped by
//                   delta = m - m' (cross_terms_pol_kernel): hh_{++} = X0 + 2 Re sum X_d e^{i d phi},
//                   hh_{xx} = W0 + 2 Re sum W_d e^{i d phi}, hh_{+x} = Y0 / 2 + Re sum Y_d e^{i d phi}
//   ln L^ML_{ikot} = dh^T [hh]^+ dh / 2                                   (Eqs. x_ML, single_det_ML)
// and, per (i, k), the maximum over (o, t) as the 64-bit key the tensor-core
// pre-selection writes (lowest t, then lowest o, on ties), so the same finish
// kernels form the per-row sums and the selection.
//
// One block per (RPB rows, detector), one thread per time slot (time chunks of
// PP_NT): the rows' components stream through shared memory in bin chunks and
// each thread accumulates the RPB x M x 2 complex Z of its time; the time-grid
// operand is the pre-selection's FP32 G, transposed to [D][B][n_tpad] (times
// innermost: a warp's loads are coalesced), or with relative binning (App. A)
// one per (mode, polarisation) component j = 2m + p, [2M][D][B][n_tpad], from
// the component weights W^{<d|h>}_{k j b}.
#include "common.cuh"
#include "kernels.h"

namespace dotpe {

namespace {
constexpr int PP_NT = 128;   // threads = time slots per pass
constexpr int PP_RPB = 4;    // bank rows per block
constexpr int PP_BCH = 64;   // bins per shared-memory chunk
}  // namespace

template <bool RB>
__global__ void __launch_bounds__(PP_NT) presel_pol_kernel(const PreselPolArgs a) {
  __shared__ __align__(16) float2 hs[PP_RPB][MAXM][2][PP_BCH];
  __shared__ float4 tab[PP_RPB][PS_MAXPHI];    // (a, 2b, c): ln L^ML = a dp^2 + 2b dp dx + c dx^2
  __shared__ float2 ph[PS_MAXPHI][MAXM];       // e^{i m phi_o}
  const int tid = threadIdx.x;
  // the detector is the fastest block index: the D blocks of one row group run
  // together and share the rows' FP32 components in L2
  const int k = (int)(blockIdx.x % (unsigned)a.n_det);
  const int64_t r0 = (int64_t)(blockIdx.x / (unsigned)a.n_det) * PP_RPB;
  const int M = a.n_modes, B = a.n_bins, D = a.n_det, np = a.n_phi;
  // phase factors (angles reduced in integers first)
  for (int q = tid; q < PS_MAXPHI * MAXM; q += PP_NT) {
    const int o = q / MAXM, m = q % MAXM;
    float s = 0.f, c = 1.f;
    if (o < np && m < M) sincospif(2.0f * (float)((a.mode_m[m] * o) % np) / (float)np, &s, &c);
    ph[o][m] = make_float2(c, s);
  }
  // [hh]^+ / 2 of the block's rows on every phase, from the rows' records
  for (int q = tid; q < PP_RPB * PS_MAXPHI; q += PP_NT) {
    const int r = q / PS_MAXPHI, o = q % PS_MAXPHI;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r0 + r < a.n_rows && o < np) {
      const float *rec = a.mx + ((r0 + r) * D + k) * REC_P;
      float A = __ldg(rec), Bx = 0.5f * __ldg(rec + 1), C = __ldg(rec + 2);
#pragma unroll
      for (int dl = 0; dl < 3; ++dl) {
        float s, c;
        sincospif(2.0f * (float)(((dl + 1) * o) % np) / (float)np, &s, &c);
        const float *g = rec + 3 + 6 * dl;
        A += 2.f * (__ldg(g) * c - __ldg(g + 1) * s);
        Bx += __ldg(g + 2) * c - __ldg(g + 3) * s;
        C += 2.f * (__ldg(g + 4) * c - __ldg(g + 5) * s);
      }
      const float det = A * C - Bx * Bx;
      if (det > a.rank_tol * A * C) {
        const float inv = 0.5f / det;
        v = make_float4(C * inv, -2.f * Bx * inv, A * inv, 0.f);
      } else if (A > 0.f || C > 0.f) {
        const float sm = A + C;
        const float inv = 0.5f / (sm * sm);
        v = make_float4(A * inv, 2.f * Bx * inv, C * inv, 0.f);
      }
    }
    tab[r][o] = v;
  }
  for (int t0 = 0; t0 < a.n_t; t0 += PP_NT) {
    const int t = t0 + tid;
    const bool tv = t < a.n_t;
    float zr[PP_RPB][MAXM][2], zi[PP_RPB][MAXM][2];
#pragma unroll
    for (int r = 0; r < PP_RPB; ++r)
#pragma unroll
      for (int m = 0; m < MAXM; ++m)
#pragma unroll
        for (int p = 0; p < 2; ++p) { zr[r][m][p] = 0.f; zi[r][m][p] = 0.f; }
    const int64_t TP = a.n_tpad;
    const float2 *g = a.G + (int64_t)k * B * TP + (tv ? t : 0);
    const int64_t gstride = (int64_t)D * B * TP;  // between components (relative binning)
    for (int b0 = 0; b0 < B; b0 += PP_BCH) {
      __syncthreads();  // the previous chunk is consumed (and, first time, the tables are written)
      for (int q = tid; q < PP_RPB * MAXM * 2 * PP_BCH; q += PP_NT) {
        const int bb = q % PP_BCH, rest = q / PP_BCH;
        const int p = rest % 2, m = (rest / 2) % MAXM, r = rest / (2 * MAXM);
        float2 v = make_float2(0.f, 0.f);
        if (r0 + r < a.n_rows && m < M && b0 + bb < B) {
          const float *row = a.master + ((int64_t)m * a.bank_rows + a.row0 + r0 + r) * a.kpad + 2 * p * B;
          v = make_float2(__ldg(row + b0 + bb), __ldg(row + B + b0 + bb));
        }
        hs[r][m][p][bb] = v;
      }
      __syncthreads();
      if (tv) {
        const int nb = min(PP_BCH, B - b0);
        // two bins per step: the rows' components of both in one 16-byte shared
        // load (bins past the chunk's end hold zeros), the operand's of both
        // loaded before either is used
        for (int bb = 0; bb < nb; bb += 2) {
          const bool two = bb + 1 < nb;
          float2 gv[2][MAXM][2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const bool in = u == 0 || two;
            if constexpr (RB) {
#pragma unroll
              for (int m = 0; m < MAXM; ++m)
#pragma unroll
                for (int p = 0; p < 2; ++p)
                  gv[u][m][p] = (m < M && in) ? __ldg(g + (2 * m + p) * gstride + (b0 + bb + u) * TP)
                                              : make_float2(0.f, 0.f);
            } else {
              const float2 g0 = in ? __ldg(g + (b0 + bb + u) * TP) : make_float2(0.f, 0.f);
#pragma unroll
              for (int m = 0; m < MAXM; ++m) gv[u][m][0] = gv[u][m][1] = g0;
            }
          }
#pragma unroll
          for (int r = 0; r < PP_RPB; ++r)
#pragma unroll
            for (int m = 0; m < MAXM; ++m)
#pragma unroll
              for (int p = 0; p < 2; ++p) {
                const float4 h2 = *reinterpret_cast<const float4 *>(&hs[r][m][p][bb]);
                const float2 g0 = gv[0][m][p], g1 = gv[1][m][p];
                zr[r][m][p] = fmaf(g0.x, h2.x, fmaf(-g0.y, h2.y, zr[r][m][p]));
                zi[r][m][p] = fmaf(g0.x, h2.y, fmaf(g0.y, h2.x, zi[r][m][p]));
                zr[r][m][p] = fmaf(g1.x, h2.z, fmaf(-g1.y, h2.w, zr[r][m][p]));
                zi[r][m][p] = fmaf(g1.x, h2.w, fmaf(g1.y, h2.z, zi[r][m][p]));
              }
        }
      }
    }
    // per row: best (ln L^ML, o) over the phases of this time, the warp's best
    // over its times, one atomic per warp
    const int lane = tid & 31;
#pragma unroll
    for (int r = 0; r < PP_RPB; ++r) {
      unsigned long long key = 0ull;
      if (tv && r0 + r < a.n_rows) {
        float best = -1.f;
        int bo = 0;
        for (int o = 0; o < np; ++o) {
          float dp = 0.f, dx = 0.f;
#pragma unroll
          for (int m = 0; m < MAXM; ++m) {
            const float2 e = ph[o][m];
            dp += zr[r][m][0] * e.x - zi[r][m][0] * e.y;
            dx += zr[r][m][1] * e.x - zi[r][m][1] * e.y;
          }
          const float4 T = tab[r][o];
          const float qv = fmaf(dp, fmaf(T.y, dx, T.x * dp), T.z * dx * dx);
          if (qv > best) { best = qv; bo = o; }
        }
        key = ((unsigned long long)__float_as_uint(fmaxf(best, 0.f)) << 32) |
              (unsigned long long)(0xffffffffu - (uint32_t)(t * np + bo));
      }
#pragma unroll
      for (int sh = 16; sh > 0; sh >>= 1) {
        const unsigned long long o2 = __shfl_xor_sync(0xffffffffu, key, sh);
        key = o2 > key ? o2 : key;
      }
      if (lane == 0 && key != 0ull) atomicMax(a.keys + (r0 + r) * D + k, key);
    }
  }
}

void launch_presel_pol(const PreselPolArgs &a, cudaStream_t st) {
  const dim3 grid((unsigned)(((a.n_rows + PP_RPB - 1) / PP_RPB) * a.n_det));
  if (a.n_gcomp > 1)
    presel_pol_kernel<true><<<grid, PP_NT, 0, st>>>(a);
  else
    presel_pol_kernel<false><<<grid, PP_NT, 0, st>>>(a);
}

}  // namespace dotpe
