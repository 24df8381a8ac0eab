// Incoherent single-detector pre-selection (Sec. IV.D, App. B) on the
// 5th-generation tensor cores.
//
// For bank row i, detector k, arrival time t_{kt} and orbital phase phi_o:
//   Z_{ikmt}        = sum_b h_{im}(f_b) c_{kb} e^{-2 pi i f_b t_{kt}}     (Eq. dh_itop, per mode)
//   <d|h>_{iktop}   = Re sum_m e^{i m phi_o} K_{imp} Z_{ikmt}
//   <h|h>_{ikopp'}  = Re sum_{m,m'} K_{imp} K^*_{im'p'} e^{i (m - m') phi_o} <h_m|h_m'>_k
//   ln L^ML_{ikot}  = dh^T [hh]^+ dh / 2                                   (Eqs. x_ML, single_det_ML)
// with K_{imp} the row's polarisation factors (h_{imp} = K_{imp} h_{im}).
// The kernel keeps, per (i, k), the maximum over (o, t) and its (o, t); the
// sum over detectors and the selection window of Sec. IV.D follow in two
// small kernels.  [hh]^+ is the inverse when det > rank_tol hh_{++} hh_{xx},
// else the rank-one pseudo-inverse hh / (hh_{++} + hh_{xx})^2.
//
// Z is one real-ified complex GEMM per mode.  A = the bank's operand planes
// (the coherent kernel's); B = G_k[b, t] = c_{kb} e^{-2 pi i f_b t_{kt}}
// packed as rows [(k, t) re; (k, t) im] x [re | im], one matrix for every
// mode.  Persistent and warp-specialised like the coherent kernel:
//   warp 0      TMA producer (A tile of the mode, B tile, 2 k-blocks per stage)
//   warp 1      TMEM allocator and tcgen05.mma issuer (lane 0)
//   warps 2..9  epilogue, two warps per TMEM lane quadrant, 16 columns each
// Tile = 128 rows x 32 (k, t) columns, all modes; accumulators of mode m in
// TMEM columns [buf 256 + 64 m, +64), two buffers.  Each detector's time grid
// is padded to a multiple of 32 columns, so a tile lies in one detector.
// Work items run row block by row block (the column tiles of one row block
// are neighbours in the schedule), so each bank row block is read from HBM
// about once and then served from L2.
//
// Epilogue thread = one row, 16 time columns of the tile.  Phases are taken
// 16 at a time: for its (row, detector) the thread forms [hh]^+ / 2 of the
// 16 phases in registers, then for every column reads the mode components
// from TMEM, forms Y_{mp} = K_{mp} Z_m and evaluates dh_p and ln L^ML on each
// phase.  The accumulator buffer is released after the last phase chunk.
#include "common.cuh"
#include "kernels.h"

namespace dotpe {

namespace {
constexpr int PTI = 128;           // bank rows per tile
constexpr int PTC = PS_TC;         // (detector, time) columns per tile
constexpr int PBN = 2 * PTC;       // GEMM columns (re, im) per tile
constexpr int PBK = 64;
constexpr int PKBX = PS_KBX;       // k-blocks per stage
constexpr int PNEPI = 8;           // epilogue warps
constexpr int PNT = (2 + PNEPI) * 32;
constexpr int PHALF = PTC / 2;     // columns per epilogue thread and tile
constexpr int OCH = 16;            // phases per register chunk
constexpr uint32_t PA_BYTES = PTI * PBK * 2, PB_BYTES = PBN * PBK * 2;
template <bool SPLIT> struct PPipe {
  static constexpr int NPL = SPLIT ? 2 : 1;
  static constexpr int ST = SPLIT ? 2 : 4;
  static constexpr uint32_t A_ST = PKBX * PA_BYTES, B_ST = PKBX * PB_BYTES;
  static constexpr uint32_t STAGE = NPL * (A_ST + B_ST);
};
constexpr uint32_t P_TMEM_COLS = 512, P_BUF_COLS = MAXM * PBN;
static_assert(2 * P_BUF_COLS <= P_TMEM_COLS, "TMEM budget");

struct PsTail {
  float4 phm[PS_MAXPHI * 2];  // (cos, sin)(m_a phi_o) of the four mode slots: [o][(c0, s0, c1, s1), (c2, s2, c3, s3)]
  float2 phd[PS_MAXPHI * 4];  // (cos, sin)(delta phi_o), delta = 0..3: [o][delta]
  uint64_t full[4], empty[4], tfull[2], tempty[2], drain;
  uint32_t tmem_slot;
  int abort_flag;
};
template <bool SPLIT>
constexpr size_t ps_smem_bytes() {
  return 1024 + (size_t)PPipe<SPLIT>::ST * PPipe<SPLIT>::STAGE + sizeof(PsTail);
}
static_assert(ps_smem_bytes<true>() <= 232448 && ps_smem_bytes<false>() <= 232448, "shared memory budget");

__device__ __forceinline__ void tmem_ld2p(uint32_t taddr, float &a, float &b) {
  uint32_t r0, r1;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(taddr));
  a = __uint_as_float(r0);
  b = __uint_as_float(r1);
}
}  // namespace

template <bool BF16, bool SPLIT>
__global__ void __launch_bounds__(PNT, 1)
    presel_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                  const __grid_constant__ PreselParams P) {
  constexpr int ST = PPipe<SPLIT>::ST, NPL = PPipe<SPLIT>::NPL;
  constexpr uint32_t STAGE_BYTES = PPipe<SPLIT>::STAGE, A_ST = PPipe<SPLIT>::A_ST, B_ST = PPipe<SPLIT>::B_ST;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *sA = base;
  uint8_t *sB = base + ST * NPL * A_ST;
  PsTail &T = *reinterpret_cast<PsTail *>(base + (size_t)ST * STAGE_BYTES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int M = P.n_modes;
  const int n_work = P.n_itile * P.n_ctile;
  const int nst = (P.kb + PKBX - 1) / PKBX;
  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(&T.full[s], 1);
      mbar_init(&T.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&T.tfull[b], 1);
      mbar_init(&T.tempty[b], PNEPI);
    }
    mbar_init(&T.drain, 1);
    T.abort_flag = 0;
    mbar_fence_init();
  }
  // phase tables (angles reduced in integers first: equal phases, equal values)
  for (int q = threadIdx.x; q < PS_MAXPHI * 4; q += PNT) {
    const int o = q >> 2, s = q & 3;
    float c = 1.f, sn = 0.f, c2 = 1.f, s2 = 0.f;
    if (o < P.n_phi) {
      const int mm = s < M ? P.mode_m[s] : 0;
      sincospif(2.0f * (float)((mm * o) % P.n_phi) / (float)P.n_phi, &sn, &c);
      sincospif(2.0f * (float)((s * o) % P.n_phi) / (float)P.n_phi, &s2, &c2);
    }
    float *pm = reinterpret_cast<float *>(&T.phm[o * 2]);
    pm[2 * s] = c;
    pm[2 * s + 1] = sn;
    T.phd[o * 4 + s] = make_float2(c2, s2);
  }
  if (warp == 0 && lane == 0) {
    tma_prefetch_desc(&mapA);
    tma_prefetch_desc(&mapB);
  }
  if (warp == 1) tmem_alloc(&T.tmem_slot, P_TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = T.tmem_slot;
  volatile int *abortp = &T.abort_flag;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      uint32_t q = 0;
      bool ok = true;
      for (int w = blockIdx.x; w < n_work && ok; w += gridDim.x) {
        const int it = w / P.n_ctile, ct = w - it * P.n_ctile;
        const int brow = ct * PBN;
        for (int m = 0; m < M && ok; ++m) {
          const int arow = m * P.a_mode_rows + P.a_row0 + it * PTI;
          for (int ks = 0; ks < nst; ++ks, ++q) {
            const int s = q % ST;
            const uint32_t n = q / ST;
            if (n > 0 && !(ok = mbar_wait(&T.empty[s], (n - 1) & 1, nullptr, abortp, P.wait_ns))) break;
            mbar_expect_tx(&T.full[s], STAGE_BYTES);
#pragma unroll
            for (int pl = 0; pl < NPL; ++pl) {
              tma_load_3d(sA + (s * NPL + pl) * A_ST, &mapA, &T.full[s], 0, pl * P.a_plane_rows + arow, ks * PKBX);
              tma_load_3d(sB + (s * NPL + pl) * B_ST, &mapB, &T.full[s], 0, pl * P.b_plane_rows + brow, ks * PKBX);
            }
          }
        }
      }
      if (!ok) {
        // let copies already in flight land before the CTA exits
        uint32_t first = q > (uint32_t)ST ? q - ST : 0;
        for (uint32_t j = first; j < q; ++j) {
          volatile int no_abort = 0;
          mbar_wait(&T.full[j % ST], (j / ST) & 1, nullptr, &no_abort, 200000000ull);
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    constexpr uint32_t idesc = idesc_f16(128, PBN, BF16);
    const bool issuer = (lane == 0);
    uint32_t q = 0, u = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < n_work && ok; w += gridDim.x) {
      const int b = u & 1;
      const uint32_t use = u >> 1;
      ++u;
      if (use > 0) ok = __all_sync(0xffffffffu, mbar_wait(&T.tempty[b], (use - 1) & 1, nullptr, abortp, P.wait_ns));
      if (!ok) break;
      tc_fence_after();
      for (int m = 0; m < M && ok; ++m) {
        const uint32_t dcol = tmem + b * P_BUF_COLS + m * PBN;
        for (int ks = 0; ks < nst; ++ks, ++q) {
          const int s = q % ST;
          const uint32_t n = q / ST;
          ok = __all_sync(0xffffffffu, mbar_wait(&T.full[s], n & 1, nullptr, abortp, P.wait_ns));
          if (!ok) break;
          tc_fence_after();
          if (issuer) {
#pragma unroll
            for (int kx = 0; kx < PKBX; ++kx) {
              const uint64_t ah = sdesc_k128(sA + (s * NPL) * A_ST + kx * PA_BYTES);
              const uint64_t bh = sdesc_k128(sB + (s * NPL) * B_ST + kx * PB_BYTES);
              const uint64_t al = sdesc_k128(sA + (s * NPL + NPL - 1) * A_ST + kx * PA_BYTES);
              const uint64_t bl = sdesc_k128(sB + (s * NPL + NPL - 1) * B_ST + kx * PB_BYTES);
#pragma unroll
              for (int k = 0; k < PBK / 16; ++k) {
                tc_mma(dcol, ah + 2 * k, bh + 2 * k, idesc, (ks | kx | k) ? 1u : 0u);
                if (SPLIT) {
                  tc_mma(dcol, ah + 2 * k, bl + 2 * k, idesc, 1u);  // hi * lo
                  tc_mma(dcol, al + 2 * k, bh + 2 * k, idesc, 1u);  // lo * hi
                }
              }
            }
            tc_commit(&T.empty[s]);
          }
          __syncwarp();
        }
      }
      if (ok && issuer) tc_commit(&T.tfull[b]);
      __syncwarp();
    }
    if (issuer) tc_commit(&T.drain);
    __syncwarp();
    volatile int no_abort = 0;
    mbar_wait(&T.drain, 0, nullptr, &no_abort, 500000000ull);
  } else {
    // ---------------- epilogue ----------------
    const int ew = warp - 2;
    const int quad = warp & 3;
    const int half = ew >> 2;
    const int row = quad * 32 + lane;
    const float zs = P.z_scale / (P.g_scale ? *P.g_scale : 1.f);
    float Kr[MAXM][2], Ki[MAXM][2];
    int cur_it = -1;
    uint32_t u = 0;
    for (int w = blockIdx.x; w < n_work; w += gridDim.x) {
      const int it = w / P.n_ctile, ct = w - it * P.n_ctile;
      const int b = u & 1;
      const uint32_t use = u >> 1;
      ++u;
      const int64_t i = (int64_t)it * PTI + row;
      const bool vi = i < P.n_rows;
      const int c0 = ct * PTC;
      const int k = c0 / P.n_tpad;
      const int t0 = c0 - k * P.n_tpad + half * PHALF;
      if (it != cur_it) {
#pragma unroll
        for (int m = 0; m < MAXM; ++m) {
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
          if (vi && m < M) v = __ldg(reinterpret_cast<const float4 *>(P.pol + (i * M + m) * 2));
          Kr[m][0] = v.x; Ki[m][0] = v.y; Kr[m][1] = v.z; Ki[m][1] = v.w;
        }
        cur_it = it;
      }
      // <h|h>_{pp'}(phi) = Dc_r + sum_delta Re(Q_r[delta] e^{i delta phi}), r = (++, +x, xx)
      float Dc[3], Qr[3][3], Qi[3][3];
      {
        float rec[REC];
        const float4 *src = reinterpret_cast<const float4 *>(P.mx + (i * P.n_det + k) * REC);
#pragma unroll
        for (int q = 0; q < REC / 4; ++q) {
          float4 v = vi ? __ldg(src + q) : make_float4(0.f, 0.f, 0.f, 0.f);
          rec[4 * q] = v.x; rec[4 * q + 1] = v.y; rec[4 * q + 2] = v.z; rec[4 * q + 3] = v.w;
        }
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const int p = r == 2 ? 1 : 0, pp = r == 0 ? 0 : 1;
          float d = 0.f;
#pragma unroll
          for (int m = 0; m < MAXM; ++m) d += rec[m] * (Kr[m][p] * Kr[m][pp] + Ki[m][p] * Ki[m][pp]);
          Dc[r] = d;
#pragma unroll
          for (int dl = 0; dl < 3; ++dl) { Qr[r][dl] = 0.f; Qi[r][dl] = 0.f; }
          int pr = 0;
#pragma unroll
          for (int a = 1; a < MAXM; ++a)
#pragma unroll
            for (int c = 0; c < a; ++c, ++pr) {
              if (a >= M) continue;
              // X = K_ap K_cp'^* + K_ap' K_cp^*
              const float xr = Kr[a][p] * Kr[c][pp] + Ki[a][p] * Ki[c][pp] + Kr[a][pp] * Kr[c][p] + Ki[a][pp] * Ki[c][p];
              const float xi = Ki[a][p] * Kr[c][pp] - Kr[a][p] * Ki[c][pp] + Ki[a][pp] * Kr[c][p] - Kr[a][pp] * Ki[c][p];
              const float hr = rec[4 + 2 * pr], hi = rec[5 + 2 * pr];
              const int dl = P.pdelta[pr] - 1;  // 0..2
              const float qr = hr * xr - hi * xi, qi = hr * xi + hi * xr;
#pragma unroll
              for (int z = 0; z < 3; ++z)
                if (z == dl) { Qr[r][z] += qr; Qi[r][z] += qi; }
            }
        }
      }
      if (!mbar_wait(&T.tfull[b], use & 1, nullptr, abortp, P.wait_ns)) break;
      tc_fence_after();
      const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + b * P_BUF_COLS;
      float best = -1.f;
      uint32_t bidx = 0xffffffffu;
      const int nch = (P.n_phi + OCH - 1) / OCH;
#pragma unroll 1
      for (int ch = 0; ch < nch; ++ch) {
        // [hh]^+ / 2 on this chunk's phases
        float ha[OCH], hb[OCH], hc[OCH];
#pragma unroll
        for (int oo = 0; oo < OCH; ++oo) {
          const int o = ch * OCH + oo;
          float hh[3];
#pragma unroll
          for (int r = 0; r < 3; ++r) hh[r] = Dc[r];
#pragma unroll
          for (int dl = 0; dl < 3; ++dl) {
            const float2 e = T.phd[o * 4 + dl + 1];
#pragma unroll
            for (int r = 0; r < 3; ++r) hh[r] += Qr[r][dl] * e.x - Qi[r][dl] * e.y;
          }
          const float A = hh[0], B = hh[1], C = hh[2];
          const float det = A * C - B * B;
          float a = 0.f, bb = 0.f, c = 0.f;
          if (det > P.rank_tol * A * C) {
            const float inv = 0.5f / det;
            a = C * inv; bb = -B * inv; c = A * inv;
          } else if (A > 0.f || C > 0.f) {
            const float s = A + C;
            const float inv = 0.5f / (s * s);
            a = A * inv; bb = B * inv; c = C * inv;
          }
          ha[oo] = a; hb[oo] = 2.f * bb; hc[oo] = c;
        }
#pragma unroll 1
        for (int j = 0; j < PHALF; ++j) {
          const int col = half * PHALF + j;
          const int t = t0 + j;
          float Zr[MAXM], Zi[MAXM];
#pragma unroll
          for (int m = 0; m < MAXM; ++m) {
            if (m < M) tmem_ld2p(tbase + m * PBN + 2 * col, Zr[m], Zi[m]);
            else { Zr[m] = 0.f; Zi[m] = 0.f; }
          }
          tmem_ld_wait();
          if (ch == nch - 1 && j == PHALF - 1) {
            // the last read of this buffer by this warp: release it to the MMA warp
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&T.tempty[b]);
          }
          if (t >= P.n_t) continue;  // padding column (warp-uniform)
          float Yr[MAXM][2], Yi[MAXM][2];
#pragma unroll
          for (int m = 0; m < MAXM; ++m) {
            const float zr = Zr[m] * zs, zi = Zi[m] * zs;
#pragma unroll
            for (int p = 0; p < 2; ++p) {
              Yr[m][p] = Kr[m][p] * zr - Ki[m][p] * zi;
              Yi[m][p] = Kr[m][p] * zi + Ki[m][p] * zr;
            }
          }
#pragma unroll
          for (int oo = 0; oo < OCH; ++oo) {
            const int o = ch * OCH + oo;
            const float4 e01 = T.phm[o * 2], e23 = T.phm[o * 2 + 1];
            float dp = e01.x * Yr[0][0] - e01.y * Yi[0][0];
            float dx = e01.x * Yr[0][1] - e01.y * Yi[0][1];
            dp = fmaf(e01.z, Yr[1][0], fmaf(-e01.w, Yi[1][0], dp));
            dx = fmaf(e01.z, Yr[1][1], fmaf(-e01.w, Yi[1][1], dx));
            dp = fmaf(e23.x, Yr[2][0], fmaf(-e23.y, Yi[2][0], dp));
            dx = fmaf(e23.x, Yr[2][1], fmaf(-e23.y, Yi[2][1], dx));
            dp = fmaf(e23.z, Yr[3][0], fmaf(-e23.w, Yi[3][0], dp));
            dx = fmaf(e23.z, Yr[3][1], fmaf(-e23.w, Yi[3][1], dx));
            const float q = fmaf(dp, fmaf(hb[oo], dx, ha[oo] * dp), hc[oo] * dx * dx);
            if (o < P.n_phi && q > best) {
              best = q;
              bidx = (uint32_t)(t * P.n_phi + o);
            }
          }
        }
      }
      if (vi && best >= -0.5f) {
        // ln L^ML >= 0: a rounding below zero counts as zero
        const unsigned long long key =
            ((unsigned long long)__float_as_uint(fmaxf(best, 0.f)) << 32) | (unsigned long long)(0xffffffffu - bidx);
        atomicMax(P.keys + i * P.n_det + k, key);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, P_TMEM_COLS);
  if (threadIdx.x == 0 && T.abort_flag) atomicCAS(P.status, 0, DEV_E_TIMEOUT);
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

template <bool BF16, bool SPLIT>
static cudaError_t launch_presel_variant(const CUtensorMap &mapA, const CUtensorMap &mapB, const PreselParams &p,
                                         int grid, cudaStream_t st) {
  auto kern = presel_kernel<BF16, SPLIT>;
  const size_t smem = ps_smem_bytes<SPLIT>();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, PNT, smem, st>>>(mapA, mapB, p);
  return cudaGetLastError();
}

int launch_presel(const CUtensorMap &mapA, const CUtensorMap &mapB, const PreselParams &p, bool bf16, bool split,
                  int n_sms, cudaStream_t st) {
  const int total = p.n_itile * p.n_ctile;
  const int grid = total < n_sms ? (total > 0 ? total : 1) : n_sms;
  cudaError_t e;
  if (bf16) e = split ? launch_presel_variant<true, true>(mapA, mapB, p, grid, st)
                      : launch_presel_variant<true, false>(mapA, mapB, p, grid, st);
  else e = split ? launch_presel_variant<false, true>(mapA, mapB, p, grid, st)
                 : launch_presel_variant<false, false>(mapA, mapB, p, grid, st);
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
