// K4 on the tensor cores: the <h|h> contraction of Eq. hh_ieo as a GEMM, used
// as a per-pair bound by the screening pass.
//
// For every pair (i, e) the coefficients of <h|h>(phi) = C_0 + 2 Re sum_delta
// C_delta e^{i delta phi} are bilinear in the row record of i (the bank's
// overlaps <h_a|h_b>_d per detector) and the column record of e
// (R_{e,d,a} R*_{e,d,b}): C_0 = sum_{d,m} M_d[mm] Q_d[mm], C_delta = sum_d
// sum_{a>b, m_a - m_b = delta} M_d[ab] Q_d[ab].  With the row record as the A
// row ([d][16] real entries, K = 48 padded to 64) and seven B rows per sample
// (C_0, Re and Im of C_1..C_3: each the column record's entries placed and
// signed so that the real product gives that output), one real GEMM of M = 128
// bank rows by N = 7 x 32 samples per tile gives every coefficient.  Both
// operands are split into bf16 hi + lo planes and multiplied in three passes
// (hi*hi + hi*lo + lo*hi, error ~2^-16 of the terms).  The epilogue forms the
// lower bound of <h|h> at every phase,
//   hmin = C_0 - 2 sum_delta |C_delta| - 2^-8 C_0
// (the last term covers the split products' rounding many times over: the
// off-diagonal terms of a Gram matrix are bounded by the diagonal ones), and
// stores it as bf16 truncated (rounded down where positive; a value that is
// not positive stays so, and the screen then rejects nothing on it).
//
// Persistent, warp-specialised like the fused kernel: warp 0 loads the tiles
// with TMA (the sample tile once per work unit of up to 64 bank tiles, the bank
// tiles through a 3-stage ring), warp 1 allocates TMEM and issues the MMAs
// into two accumulator buffers of 224 columns, warps 2-17 read the
// accumulators (four warps per TMEM lane quadrant, 8 samples each), form the
// bounds and store them.  Every wait is bounded.
#include "common.cuh"
#include "kernels.h"

namespace dotpe {

namespace {
constexpr int HB_TI = 128;               // bank rows per tile (M)
constexpr int HB_TE = 32;                // extrinsic samples per tile
constexpr int HB_NC = 7;                 // outputs per sample: C_0, Re/Im C_1..C_3
constexpr int HB_BN = HB_TE * HB_NC;     // 224 B rows per tile: N of each MMA
constexpr int HB_K = 64;                 // K: 3 detectors x 16 record entries, padded
constexpr int HB_ST = 3;                 // bank-tile stages
constexpr int HB_NEPI = 16;              // epilogue warps (four per TMEM lane quadrant, 8 samples each)
constexpr int HB_NT = (2 + HB_NEPI) * 32;
constexpr int HB_CHUNK = 64;             // bank tiles per work unit
constexpr uint32_t HB_A_BYTES = HB_TI * HB_K * 2;  // one plane of a bank tile (16 KB)
constexpr uint32_t HB_B_BYTES = HB_BN * HB_K * 2;  // one plane of a sample tile (28 KB)
constexpr uint32_t HB_TMEM_COLS = 512, HB_BUF = 256;
static_assert(HB_A_BYTES % 1024 == 0 && HB_B_BYTES % 1024 == 0, "1024-byte aligned planes");

struct HbSmem {
  uint8_t A[HB_ST][2][HB_A_BYTES];
  uint8_t B[2][HB_B_BYTES];
  uint64_t full[HB_ST], empty[HB_ST], bfull, bfree, tfull[2], tempty[2], drain;
  uint32_t tmem_slot;
  int abort_flag;
};
constexpr size_t HB_SMEM = 1024 + sizeof(HbSmem);
static_assert(HB_SMEM <= 232448, "shared memory budget");


// 32 lanes x 32-bit, 8 consecutive columns per thread.
__device__ __forceinline__ void hb_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = __uint_as_float(r[k]);
}
}  // namespace

// Row-record planes [2][rows_pad][64] bf16 (hi, lo) of a block's row records
// mx [rows][D][16]: entry k = d * 16 + r, zero beyond the detectors and rows.
__global__ void hb_pack_rows_kernel(int64_t rows, int64_t rows_pad, int D, const float *__restrict__ mx,
                                    __nv_bfloat16 *__restrict__ out) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= rows_pad * HB_K) return;
  const int64_t i = q / HB_K;
  const int k = (int)(q % HB_K), d = k / REC, r = k % REC;
  const float v = (i < rows && d < D) ? mx[(i * D + d) * REC + r] : 0.f;
  const __nv_bfloat16 hi = __float2bfloat16_rn(v);
  out[q] = hi;
  out[rows_pad * HB_K + q] = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// Sample planes [2][n_etile * 224][64] bf16 (hi, lo): row (et, s, c) of sample
// e = 32 et + s and output c; entry k = d * 16 + r as for the rows.
__global__ void hb_pack_cols_kernel(int64_t E, int n_etile, int D, HbDelta dl, const float *__restrict__ qx,
                                    __nv_bfloat16 *__restrict__ out) {
  const int64_t total = (int64_t)n_etile * HB_BN * HB_K;
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= total) return;
  const int64_t row = q / HB_K;
  const int k = (int)(q % HB_K), d = k / REC, r = k % REC;
  const int64_t e = (row / HB_BN) * HB_TE + (row % HB_BN) / HB_NC;
  const int c = (int)(row % HB_NC);
  float v = 0.f;
  if (e < E && d < D) {
    const float *rec = qx + (e * D + d) * REC;
    if (c == 0) {
      if (r < MAXM) v = rec[r];  // C_0: the diagonal entries
    } else if (r >= MAXM) {
      const int delta = (c + 1) / 2, im = (c % 2 == 0);
      const int p = (r - MAXM) / 2, part = (r - MAXM) % 2;  // part 0: Re M_ab slot, 1: Im M_ab slot
      if (p < NPAIR && dl.pdelta[p] == delta) {
        const float qr = rec[MAXM + 2 * p], qi = rec[MAXM + 2 * p + 1];
        // Re(M Q) = Mr Qr - Mi Qi, Im(M Q) = Mr Qi + Mi Qr
        v = im ? (part == 0 ? qi : qr) : (part == 0 ? qr : -qi);
      }
    }
  }
  const __nv_bfloat16 hi = __float2bfloat16_rn(v);
  out[q] = hi;
  out[total + q] = __float2bfloat16_rn(v - __bfloat162float(hi));
}

__global__ void __launch_bounds__(HB_NT, 1)
    hb_bound_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, HbArgs a) {
  extern __shared__ uint8_t smem_raw[];
  HbSmem &S = *reinterpret_cast<HbSmem *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_chunk = (a.n_itile + HB_CHUNK - 1) / HB_CHUNK;
  const int n_units = a.n_etile * n_chunk;
  const unsigned long long wait_ns = 4000000000ull;
  if (threadIdx.x == 0) {
    for (int s = 0; s < HB_ST; ++s) {
      mbar_init(&S.full[s], 1);
      mbar_init(&S.empty[s], 1);
    }
    mbar_init(&S.bfull, 1);
    mbar_init(&S.bfree, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&S.tfull[b], 1);
      mbar_init(&S.tempty[b], HB_NEPI);
    }
    mbar_init(&S.drain, 1);
    S.abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == 0 && lane == 0) {
    tma_prefetch_desc(&mapA);
    tma_prefetch_desc(&mapB);
  }
  if (warp == 1) tmem_alloc(&S.tmem_slot, HB_TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem_slot;
  volatile int *abortp = &S.abort_flag;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      uint32_t q = 0, nb = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x, ++nb) {
        const int et = u / n_chunk, c = u % n_chunk;
        if (nb > 0 && !(ok = mbar_wait(&S.bfree, (nb - 1) & 1, nullptr, abortp, wait_ns))) break;
        mbar_expect_tx(&S.bfull, 2 * HB_B_BYTES);
        for (int pl = 0; pl < 2; ++pl)
          tma_load_3d(S.B[pl], &mapB, &S.bfull, 0, pl * a.b_plane_rows + et * HB_BN, 0);
        const int it1 = min(a.n_itile, (c + 1) * HB_CHUNK);
        for (int it = c * HB_CHUNK; it < it1; ++it, ++q) {
          const int s = q % HB_ST;
          const uint32_t n = q / HB_ST;
          if (n > 0 && !(ok = mbar_wait(&S.empty[s], (n - 1) & 1, nullptr, abortp, wait_ns))) break;
          mbar_expect_tx(&S.full[s], 2 * HB_A_BYTES);
          for (int pl = 0; pl < 2; ++pl)
            tma_load_3d(S.A[s][pl], &mapA, &S.full[s], 0, pl * a.a_plane_rows + it * HB_TI, 0);
        }
      }
      if (!ok) {
        // let copies already in flight land before the CTA exits
        uint32_t first = q > (uint32_t)HB_ST ? q - HB_ST : 0;
        for (uint32_t j = first; j < q; ++j) {
          volatile int no_abort = 0;
          mbar_wait(&S.full[j % HB_ST], (j / HB_ST) & 1, nullptr, &no_abort, 200000000ull);
        }
        volatile int no_abort = 0;
        if (nb > 0) mbar_wait(&S.bfull, (nb - 1) & 1, nullptr, &no_abort, 200000000ull);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    constexpr uint32_t idesc = idesc_f16(128, HB_BN, true);
    const bool issuer = (lane == 0);
    uint32_t q = 0, u2 = 0, nb = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x, ++nb) {
      const int c = u % n_chunk;
      ok = __all_sync(0xffffffffu, mbar_wait(&S.bfull, nb & 1, nullptr, abortp, wait_ns));
      if (!ok) break;
      tc_fence_after();
      const int it1 = min(a.n_itile, (c + 1) * HB_CHUNK);
      for (int it = c * HB_CHUNK; it < it1 && ok; ++it, ++q, ++u2) {
        const int b = u2 & 1;
        const uint32_t use = u2 >> 1;
        if (use > 0) ok = __all_sync(0xffffffffu, mbar_wait(&S.tempty[b], (use - 1) & 1, nullptr, abortp, wait_ns));
        if (!ok) break;
        const int s = q % HB_ST;
        ok = __all_sync(0xffffffffu, mbar_wait(&S.full[s], (q / HB_ST) & 1, nullptr, abortp, wait_ns));
        if (!ok) break;
        tc_fence_after();
        if (issuer) {
          const uint32_t d = tmem + b * HB_BUF;
          const uint64_t ah = sdesc_k128(S.A[s][0]), al = sdesc_k128(S.A[s][1]);
          const uint64_t bh = sdesc_k128(S.B[0]), bl = sdesc_k128(S.B[1]);
          // K steps beyond the detectors hold zeros in both operands
#pragma unroll
          for (int k = 0; k < HB_K / 16; ++k)
            if (k < a.n_kstep) {
              tc_mma(d, ah + 2 * k, bh + 2 * k, idesc, k ? 1u : 0u);  // hi * hi
              tc_mma(d, ah + 2 * k, bl + 2 * k, idesc, 1u);          // hi * lo
              tc_mma(d, al + 2 * k, bh + 2 * k, idesc, 1u);          // lo * hi
            }
          tc_commit(&S.empty[s]);
          tc_commit(&S.tfull[b]);
        }
        __syncwarp();
      }
      // the sample tile may be replaced once this unit's MMAs complete
      if (ok && issuer) tc_commit(&S.bfree);
      __syncwarp();
    }
    if (issuer) tc_commit(&S.drain);
    __syncwarp();
    volatile int no_abort = 0;
    mbar_wait(&S.drain, 0, nullptr, &no_abort, 500000000ull);
  } else {
    // ---------------- epilogue: one row, 8 samples per thread ----------------
    const int ew = warp - 2, quad = warp & 3, part = ew >> 2;
    const int row = quad * 32 + lane;
    uint32_t u2 = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
      const int et = u / n_chunk, c = u % n_chunk;
      const int it1 = min(a.n_itile, (c + 1) * HB_CHUNK);
      for (int it = c * HB_CHUNK; it < it1; ++it, ++u2) {
        const int b = u2 & 1;
        const uint32_t use = u2 >> 1;
        if (!(ok = mbar_wait(&S.tfull[b], use & 1, nullptr, abortp, wait_ns))) break;
        tc_fence_after();
        // this thread's 8 samples x 7 outputs: columns [56 part, +56)
        float v[HB_NC][8];
        const uint32_t t0 = tmem + ((uint32_t)(quad * 32) << 16) + b * HB_BUF + 56 * part;
#pragma unroll
        for (int g = 0; g < HB_NC; ++g) hb_ld8(t0 + 8 * g, v[g]);
        tmem_ld_wait();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.tempty[b]);
        // column 8 g + x of this thread's range holds sample (8 g + x) / 7, output (8 g + x) % 7
        uint32_t o[4];
#pragma unroll
        for (int sm = 0; sm < 8; sm += 2) {
          float h2[2];
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            float cc[HB_NC];
#pragma unroll
            for (int k = 0; k < HB_NC; ++k) cc[k] = v[((sm + t) * HB_NC + k) / 8][((sm + t) * HB_NC + k) % 8];
            float h = cc[0] * (1.f - 0.00390625f);
#pragma unroll
            for (int dl = 0; dl < 3; ++dl)
              h = fmaf(-2.000004f, sqrt_near(fmaf(cc[1 + 2 * dl], cc[1 + 2 * dl], cc[2 + 2 * dl] * cc[2 + 2 * dl])), h);
            h2[t] = h;
          }
          // the upper halves of the two floats: bf16 truncated, sample sm in the low half
          o[sm >> 1] = __byte_perm(__float_as_uint(h2[0]), __float_as_uint(h2[1]), 0x7632);
        }
        const int64_t i = (int64_t)it * HB_TI + row;
        if (i < a.n_rows)
          __stcs(reinterpret_cast<uint4 *>(a.out + i * a.ld + (int64_t)et * HB_TE + 8 * part),
                 make_uint4(o[0], o[1], o[2], o[3]));  // streamed: read once by the screen
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, HB_TMEM_COLS);
  if (threadIdx.x == 0 && S.abort_flag && a.status) atomicCAS(a.status, 0, DEV_E_TIMEOUT);
}

static inline unsigned hb_nblk(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

size_t hb_scratch_bytes(int64_t rows, int64_t E) {
  const int64_t rows_pad = (rows + HB_TI - 1) / HB_TI * HB_TI;
  const int64_t n_etile = (E + HB_TE - 1) / HB_TE;
  return (size_t)(2 * rows_pad * HB_K * 2) + 256 + (size_t)(2 * n_etile * HB_BN * HB_K * 2) + 256 +
         (size_t)(rows_pad * hb_ld(E) * 2) + 256;
}

// row stride of the bound: a multiple of 64 samples, so that a 64-sample
// screening tile reads whole 16-byte words inside the row
int64_t hb_ld(int64_t E) { return (E + 63) / 64 * 64; }

int launch_hh_bound(int64_t rows, int64_t E, int D, const HbDelta &dl, const float *mx, const float *qx,
                    void *scratch, __nv_bfloat16 **out, int n_sms, int *status, cudaStream_t st) {
  if (D < 1 || D > MAXD || rows < 1 || E < 1) return -4;
  const int64_t rows_pad = (rows + HB_TI - 1) / HB_TI * HB_TI;
  const int n_itile = (int)(rows_pad / HB_TI), n_etile = (int)((E + HB_TE - 1) / HB_TE);
  uint8_t *p = (uint8_t *)scratch;
  __nv_bfloat16 *ra = (__nv_bfloat16 *)p;
  p += ((size_t)(2 * rows_pad * HB_K * 2) + 255) / 256 * 256;
  __nv_bfloat16 *cb = (__nv_bfloat16 *)p;
  p += ((size_t)(2 * n_etile * HB_BN * HB_K * 2) + 255) / 256 * 256;
  *out = (__nv_bfloat16 *)p;
  hb_pack_rows_kernel<<<hb_nblk(rows_pad * HB_K, 256), 256, 0, st>>>(rows, rows_pad, D, mx, ra);
  hb_pack_cols_kernel<<<hb_nblk((int64_t)n_etile * HB_BN * HB_K, 256), 256, 0, st>>>(E, n_etile, D, dl, qx, cb);
  CUtensorMap mapA, mapB;
  if (encode_tmap_kblocks(&mapA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, ra, 2 * rows_pad, 1, HB_K * 2, HB_TI, 1))
    return -1;
  if (encode_tmap_kblocks(&mapB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, cb, 2 * (int64_t)n_etile * HB_BN, 1, HB_K * 2,
                          HB_BN, 1))
    return -1;
  HbArgs a;
  a.n_rows = rows;
  a.n_itile = n_itile;
  a.n_etile = n_etile;
  a.a_plane_rows = (int)rows_pad;
  a.b_plane_rows = n_etile * HB_BN;
  a.n_kstep = D;
  a.out = *out;
  a.ld = hb_ld(E);
  a.status = status;
  if (cudaFuncSetAttribute(hb_bound_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HB_SMEM) !=
      cudaSuccess)
    return -2;
  const int n_units = n_etile * ((n_itile + HB_CHUNK - 1) / HB_CHUNK);
  const int grid = n_units < n_sms ? n_units : n_sms;
  hb_bound_kernel<<<grid, HB_NT, HB_SMEM, st>>>(mapA, mapB, a);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace dotpe
