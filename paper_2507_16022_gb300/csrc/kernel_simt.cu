// K7: plain FP32 path.  Fused <d|h> GEMM (FFMA, shared-memory tiles) and the
// marginalisation epilogue, one 64 x 32 (i, e) tile per block.
//
// Per mode m the GEMM is the real-ified complex product of Eq. dh_ieo:
//   [h_r | h_i] (K = 2B) x [(e,re): (G_r | -G_i), (e,im): (G_i | G_r)]
// so the two output columns of extrinsic sample e are Re Z_m and Im Z_m.
#include "common.cuh"
#include "epilogue.cuh"
#include "kernels.h"

namespace dotpe {

namespace {
constexpr int TI = SIMT_TI, TE = SIMT_TE, NC = 2 * TE, KC = 32, NT = 256;

struct SimtSmem {
  union {
    struct {
      float As[KC][TI + 4];
      float Bs[KC][NC + 4];
    } g;
    struct {
      float xs[TI][TE + 1], x2s[TI][TE + 1];
    } r;
  } u;
  float mls[TI][TE + 1];
  int pks[TI][TE + 1];  // argo | npass << 16
  alignas(16) float qs[TE * MAXD * REC];  // read as float4 records
  double lwe[TE];
  float2 ph[7 * MAXPHI];
  float r_m1[TI], r_s1[TI], r_m2[TI], r_s2[TI], r_ml[TI];
  long long r_arg[TI];
  int r_np[TI];
};
}

__global__ void __launch_bounds__(NT) simt_fused_kernel(SimtArgs g, EpiParams P) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  SimtSmem &S = *reinterpret_cast<SimtSmem *>(smem_raw);
  auto &As = S.u.g.As;
  auto &Bs = S.u.g.Bs;
  auto &xs = S.u.r.xs;
  auto &x2s = S.u.r.x2s;
  auto &mls = S.mls;
  auto &pks = S.pks;
  float *qs = S.qs;
  double *lwe = S.lwe;
  float2 *ph = S.ph;
  float *r_m1 = S.r_m1, *r_s1 = S.r_s1, *r_m2 = S.r_m2, *r_s2 = S.r_s2, *r_ml = S.r_ml;
  long long *r_arg = S.r_arg;
  int *r_np = S.r_np;

  const int tid = threadIdx.x;
  const int et = blockIdx.x, it = blockIdx.y;
  const int64_t i0 = (int64_t)it * TI, e0 = (int64_t)et * TE;
  const int ty = tid / 16, tx = tid % 16;

  fill_phase_tables(ph, P, tid, NT);
  for (int k = tid; k < TE * P.n_det * REC; k += NT) {
    int e = k / (P.n_det * REC), q = k % (P.n_det * REC);
    qs[e * MAXD * REC + q] = (e0 + e < P.n_ext) ? P.qx[(e0 + e) * P.n_det * REC + q] : 0.f;
  }
  for (int k = tid; k < TE; k += NT) lwe[k] = (P.lw_ext && e0 + k < P.n_ext) ? P.lw_ext[e0 + k] : 0.0;

  float acc[MAXM][4][4];
#pragma unroll
  for (int m = 0; m < MAXM; ++m)
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[m][r][c] = 0.f;

#pragma unroll
  for (int m = 0; m < MAXM; ++m) {
    if (m >= P.n_modes) break;
    const float *Abase = g.A + ((int64_t)m * g.I_bank + P.i_base + i0) * g.Kpad;
    const float *Bbase = g.Bm + ((int64_t)m * 2 * P.n_ext + 2 * e0) * g.Kpad;
#pragma unroll 1
    for (int k0 = 0; k0 < g.K; k0 += KC) {
      __syncthreads();
      // A chunk: 64 rows x 32 k -> As[k][row]
      for (int q = tid; q < TI * KC; q += NT) {
        int row = q / KC, kk = q % KC;
        float v = 0.f;
        if (i0 + row < P.n_int && k0 + kk < g.K) v = __ldg(Abase + (int64_t)row * g.Kpad + k0 + kk);
        As[kk][row] = v;
      }
      for (int q = tid; q < NC * KC; q += NT) {
        int col = q / KC, kk = q % KC;
        float v = 0.f;
        if (2 * e0 + col < 2 * P.n_ext && k0 + kk < g.K) v = __ldg(Bbase + (int64_t)col * g.Kpad + k0 + kk);
        Bs[kk][col] = v;
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < KC; ++kk) {
        float a[4], b[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) a[r] = As[kk][ty * 4 + r];
#pragma unroll
        for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx * 4 + c];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[m][r][c] = fmaf(a[r], b[c], acc[m][r][c]);
      }
    }
  }
  __syncthreads();

  const float thr = tile_threshold(P);
  const bool store = (P.lnl_tile != nullptr);
  const float zs = P.z_scale / (P.g_scale ? *P.g_scale : 1.f);
  // epilogue: 4 rows x 2 extrinsic samples per thread
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int rl = ty * 4 + r;
    const int64_t i = i0 + rl;
    const bool vi = i < P.n_int;
    float mrec[MAXD * REC];
    const bool pol = (P.n_pol == 2);
#pragma unroll
    for (int q = 0; q < MAXD * REC; ++q) mrec[q] = 0.f;
#pragma unroll
    for (int q = 0; q < MAXD * REC; ++q)
      if (vi && !pol && q < P.n_det * REC) mrec[q] = __ldg(P.mx + i * P.n_det * REC + q);
    const double lwi = (vi && P.lw_int) ? P.lw_int[i] : 0.0;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int el = tx * 2 + j;
      const int64_t e = e0 + el;
      float x = -INFINITY, x2 = -INFINITY, ml = -1.f;
      int pk = 0;
      if (vi && e < P.n_ext) {
        float Zr[MAXM], Zi[MAXM];
#pragma unroll
        for (int mm = 0; mm < MAXM; ++mm) {
          bool on = mm < P.n_modes;
          Zr[mm] = on ? acc[mm][r][2 * j] * zs : 0.f;
          Zi[mm] = on ? acc[mm][r][2 * j + 1] * zs : 0.f;
        }
        if (P.gemm_only) {
          float sx = 0.f;
#pragma unroll
          for (int mm = 0; mm < MAXM; ++mm) sx += Zr[mm] + Zi[mm];
          x = sx; x2 = sx; ml = 0.f;
        } else {
          float C0, Cr[3], Ci[3];
          if (pol) hh_coeffs_pol(P.mx + i * P.n_det * REC_P, &qs[el * MAXD * REC], P, C0, Cr, Ci);
          else hh_coeffs<false>(mrec, &qs[el * MAXD * REC], P, C0, Cr, Ci);
          PairRes pr = pair_eval(Zr, Zi, C0, Cr, Ci, thr, !store, P, ph);
          float lw = (float)(lwi + lwe[el]);
          x = pr.lsum + lw;
          x2 = pr.lsum2 + 2.f * lw;
          ml = pr.ml;
          pk = pr.argo | (pr.npass << 16);
          if (store) {
            P.lnl_tile[i * P.n_ext + e] = pr.lsum - P.ln_nphi;
            P.ml_tile[i * P.n_ext + e] = pr.ml;
          }
        }
      }
      xs[rl][el] = x;
      x2s[rl][el] = x2;
      mls[rl][el] = ml;
      pks[rl][el] = pk;
    }
  }
  __syncthreads();

  const int64_t tile = (int64_t)it * gridDim.x + et;
  if (tid < TI) {
    // row partials over the tile's extrinsic samples
    Lse a, b;
    a.init(); b.init();
    float best = -1.f;
    long long barg = 0;
    int np = 0;
    for (int c = 0; c < TE; ++c) {
      a.add(xs[tid][c]);
      b.add(x2s[tid][c]);
      int pk = pks[tid][c];
      np += pk >> 16;
      float v = mls[tid][c];
      if (v > best) { best = v; barg = ((i0 + tid) * P.n_ext + e0 + c) * (long long)P.n_phi + (pk & 0xFFFF); }
    }
    if (i0 + tid < P.n_int) P.row_part[(int64_t)et * P.n_int + i0 + tid] = make_float2(a.m, a.s);
    r_m1[tid] = a.m; r_s1[tid] = a.s; r_m2[tid] = b.m; r_s2[tid] = b.s;
    r_ml[tid] = best; r_arg[tid] = barg; r_np[tid] = np;
  } else if (tid < TI + TE) {
    const int c = tid - TI;
    Lse a;
    a.init();
    for (int rr = 0; rr < TI; ++rr) a.add(xs[rr][c]);
    if (e0 + c < P.n_ext) P.col_part[(int64_t)it * P.n_ext + e0 + c] = make_float2(a.m, a.s);
  }
  __syncthreads();
  if (tid < 32) {
    Lse a, b;
    a.init(); b.init();
    float best = -1.f;
    long long barg = 0x7fffffffffffffffLL;
    int np = 0;
    for (int rr = tid; rr < TI; rr += 32) {
      a.merge(r_m1[rr], r_s1[rr]);
      b.merge(r_m2[rr], r_s2[rr]);
      np += r_np[rr];
      if (r_ml[rr] > best || (r_ml[rr] == best && r_arg[rr] < barg)) { best = r_ml[rr]; barg = r_arg[rr]; }
    }
    warp_merge_lse(a);
    warp_merge_lse(b);
    warp_argmax(best, barg);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) np += __shfl_xor_sync(0xffffffffu, np, o);
    if (tid == 0) {
      P.tile_part[tile] = make_float4(a.m, a.s, b.m, b.s);
      P.tile_ml[tile] = best;
      P.tile_arg[tile] = barg;
      P.tile_npass[tile] = np;
      if (best > 0.f && P.track_max) atomic_max_nonneg(P.ml_running, best);
    }
  }
}

void launch_simt(const SimtArgs &g, const EpiParams &P, cudaStream_t st) {
  dim3 grid((unsigned)((P.n_ext + TE - 1) / TE), (unsigned)((P.n_int + TI - 1) / TI));
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(simt_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SimtSmem));
    attr = true;
  }
  simt_fused_kernel<<<grid, NT, sizeof(SimtSmem), st>>>(g, P);
}

}  // namespace dotpe
