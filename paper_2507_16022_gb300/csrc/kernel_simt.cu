// K7: plain FP32 path.  Fused <d|h> GEMM (FFMA on the CUDA cores) and the
// marginalisation epilogue, one 64 x 32 (i, e) tile per block.
//
// Per mode m the GEMM is the real-ified complex product of Eq. dh_ieo:
//   [h_r | h_i] (K = 2B) x [(e,re): (G_r | -G_i), (e,im): (G_i | G_r)]
// so each extrinsic sample e has two output columns, Re Z_m and Im Z_m.  The
// FP32 extrinsic operand interleaves them along K, [m][e][Kpad][2].
//
// Mainloop: K in chunks of 16, every mode's A (64 bank rows) and B (32
// samples) chunk copied into shared memory with cp.async (16-byte copies, two
// stages: the next chunk's copies overlap this chunk's FMAs).  Each thread
// accumulates 4 rows x 2 samples x (re, im) x 4 modes in registers; per k-quad
// and mode it reads 4 + 4 float4 from shared memory for 64 FMAs (the A reads
// are broadcasts, the B rows 36 words apart so that 16 lanes read 16 samples
// in two wavefronts).
#include "common.cuh"
#include "epilogue.cuh"
#include "kernels.h"

namespace dotpe {

namespace {
constexpr int TI = SIMT_TI, TE = SIMT_TE, KC = 16, NT = 256;
constexpr int AS_LD = KC + 4;      // words per bank row of a stage
constexpr int BS_LD = 2 * KC + 4;  // words per extrinsic sample of a stage ((re, im) per k)

struct SimtStage {
  float A[MAXM][TI][AS_LD];
  float B[MAXM][TE][BS_LD];
};

struct SimtSmem {
  union {
    SimtStage st[2];
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

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(smem)), "l"(gmem),
               "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
}  // namespace

__global__ void __launch_bounds__(NT, 2) simt_fused_kernel(SimtArgs g, EpiParams P) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  SimtSmem &S = *reinterpret_cast<SimtSmem *>(smem_raw);
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
  const int ty = tid / 16, tx = tid % 16;  // rows ty*4 .. ty*4+3, samples tx and tx + 16
  const int M = P.n_modes;

  fill_phase_tables(ph, P, tid, NT);
  for (int k = tid; k < TE * P.n_det * REC; k += NT) {
    int e = k / (P.n_det * REC), q = k % (P.n_det * REC);
    qs[e * MAXD * REC + q] = (e0 + e < P.n_ext) ? P.qx[(e0 + e) * P.n_det * REC + q] : 0.f;
  }
  for (int k = tid; k < TE; k += NT) lwe[k] = (P.lw_ext && e0 + k < P.n_ext) ? P.lw_ext[e0 + k] : 0.0;

  float acc[MAXM][4][2][2];
#pragma unroll
  for (int m = 0; m < MAXM; ++m)
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        acc[m][r][j][0] = 0.f;
        acc[m][r][j][1] = 0.f;
      }

  // one chunk of every mode's operands into stage s (zero-filled outside the
  // slice, the extrinsic samples and the modes)
  const int nch = (g.K + KC - 1) / KC;
  auto load_chunk = [&](int c, int s) {
    const int k0 = c * KC;
    SimtStage &st = S.u.st[s];
    for (int f = tid; f < MAXM * TI * (KC / 4); f += NT) {
      const int m = f / (TI * (KC / 4)), r = (f / (KC / 4)) % TI, q = f % (KC / 4);
      const bool ok = m < M && i0 + r < P.n_int;
      const float *src = ok ? g.A + ((int64_t)m * g.I_bank + P.i_base + i0 + r) * g.Kpad + k0 + 4 * q : g.A;
      cp_async16(&st.A[m][r][4 * q], src, ok);
    }
    for (int f = tid; f < MAXM * TE * (2 * KC / 4); f += NT) {
      const int m = f / (TE * (2 * KC / 4)), e = (f / (2 * KC / 4)) % TE, q = f % (2 * KC / 4);
      const bool ok = m < M && e0 + e < P.n_ext;
      const float *src = ok ? g.Bm + (((int64_t)m * P.n_ext + e0 + e) * g.Kpad + k0) * 2 + 4 * q : g.Bm;
      cp_async16(&st.B[m][e][4 * q], src, ok);
    }
    cp_async_commit();
  };

  load_chunk(0, 0);
#pragma unroll 1
  for (int c = 0; c < nch; ++c) {
    if (c + 1 < nch) {
      load_chunk(c + 1, (c + 1) & 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const SimtStage &st = S.u.st[c & 1];
#pragma unroll
    for (int m = 0; m < MAXM; ++m) {
      if (m >= M) break;
#pragma unroll
      for (int kq = 0; kq < KC / 4; ++kq) {
        float4 a[4], b[2][2];
#pragma unroll
        for (int r = 0; r < 4; ++r) a[r] = *reinterpret_cast<const float4 *>(&st.A[m][ty * 4 + r][4 * kq]);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          b[j][0] = *reinterpret_cast<const float4 *>(&st.B[m][tx + 16 * j][8 * kq]);
          b[j][1] = *reinterpret_cast<const float4 *>(&st.B[m][tx + 16 * j][8 * kq + 4]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            // b[j][0] = (re_k, im_k, re_k+1, im_k+1), b[j][1] the same for k+2, k+3
            float sr = acc[m][r][j][0], si = acc[m][r][j][1];
            sr = fmaf(a[r].x, b[j][0].x, sr);
            si = fmaf(a[r].x, b[j][0].y, si);
            sr = fmaf(a[r].y, b[j][0].z, sr);
            si = fmaf(a[r].y, b[j][0].w, si);
            sr = fmaf(a[r].z, b[j][1].x, sr);
            si = fmaf(a[r].z, b[j][1].y, si);
            sr = fmaf(a[r].w, b[j][1].z, sr);
            si = fmaf(a[r].w, b[j][1].w, si);
            acc[m][r][j][0] = sr;
            acc[m][r][j][1] = si;
          }
      }
    }
    __syncthreads();
  }

  const float thr = tile_threshold(P);
  const bool store = (P.lnl_tile != nullptr);
  const float zs = P.z_scale / (P.g_scale ? *P.g_scale : 1.f);
  // epilogue: 4 rows x 2 extrinsic samples per thread
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int rl = ty * 4 + r;
    const int64_t i = i0 + rl;
    const bool vi = i < P.n_int;
    // the row's records are read through the cache for each pair (registers
    // stay with the accumulators)
    const bool pol = (P.n_pol == 2);
    const float *mrow = P.mx + i * P.n_det * (pol ? REC_P : REC);
    const double lwi = (vi && P.lw_int) ? P.lw_int[i] : 0.0;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int el = tx + 16 * j;
      const int64_t e = e0 + el;
      float x = -INFINITY, x2 = -INFINITY, ml = -1.f;
      int pk = 0;
      if (vi && e < P.n_ext) {
        float Zr[MAXM], Zi[MAXM];
#pragma unroll
        for (int mm = 0; mm < MAXM; ++mm) {
          bool on = mm < P.n_modes;
          Zr[mm] = on ? acc[mm][r][j][0] * zs : 0.f;
          Zi[mm] = on ? acc[mm][r][j][1] * zs : 0.f;
        }
        if (P.gemm_only) {
          float sx = 0.f;
#pragma unroll
          for (int mm = 0; mm < MAXM; ++mm) sx += Zr[mm] + Zi[mm];
          x = sx; x2 = sx; ml = 0.f;
        } else {
          float C0, Cr[3], Ci[3];
          if (pol) hh_coeffs_pol(mrow, &qs[el * MAXD * REC], P, C0, Cr, Ci);
          else hh_coeffs<false>(mrow, &qs[el * MAXD * REC], P, C0, Cr, Ci);
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
