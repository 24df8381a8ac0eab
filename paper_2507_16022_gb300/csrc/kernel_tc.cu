// Host side of the fused tcgen05 kernel: tensor maps, L2 bands, launches of
// batches of up to TC_MAXB events (single events go through kernel_tc1.cu).
#include "kernel_tc.cuh"

namespace dotpe {

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

// 3-D view of a row-major [rows][n_kb * 64] matrix: dims {64, rows, n_kb}, box
// {64, box_rows, box_kb} -> shared memory [box_kb][box_rows][64], 128-byte swizzle.
int encode_tmap_kblocks(CUtensorMap *map, CUtensorMapDataType dt, void *base, uint64_t rows, uint64_t n_kb,
                        uint64_t row_bytes, uint32_t box_rows, uint32_t box_kb) {
  if (!g_encode) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return -1;
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  cuuint64_t dims[3] = {64, rows, n_kb};
  cuuint64_t strides[2] = {row_bytes, 128};
  cuuint32_t box[3] = {64, box_rows, box_kb};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = g_encode(map, dt, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -2;
}

int tc_kblocks_per_stage() { return KBX; }

int tc_band(double l2_band_bytes, int kb, int n_modes, bool split, int n_etile) {
  // extrinsic operand bytes of one tile column (all modes, planes)
  const double tile_bytes = 2.0 * TE * kb * BK * 2.0 * n_modes * (split ? 2 : 1);
  int band = (int)(l2_band_bytes / tile_bytes);
  return band < 1 ? 1 : (band > n_etile ? n_etile : band);
}

// Launch of one batch in a given instantiation (NB = 1 lives in kernel_tc1.cu).
template <int NB>
int launch_tc_nb(const TcLaunch &L, const TcWork *works, int n, const int2 *glist, const int *glist_n,
                 cudaStream_t st) {
  static_assert(sizeof(TcBatch<NB>) <= 32000, "kernel parameter space");
  if (n < 1 || n > NB) return (int)cudaErrorInvalidValue;
  const int tev = L.tev == 64 ? 64 : 32;
  TcBatch<NB> *bt = new TcBatch<NB>();  // ~29 KB: off the host stack
  int total = 0;
  for (int k = 0; k < n; ++k) {
    bt->w[k] = works[k];
    bt->mapB[k] = (tev == 64) ? works[k].mapB64 : works[k].mapB;
    bt->begin[k] = total;
    total += tc_work_items(works[k], tev);
  }
  for (int k = n; k <= NB; ++k) bt->begin[k] = total;
  bt->n = n;
  bt->glist = glist;
  bt->glist_n = glist_n;
  bt->gate = L.gate;
  bt->gate_want = L.gate_want;
  // a list's length is known on the device only: one CTA per SM
  int grid = (glist || L.n_sms < total) ? L.n_sms : total;
  if (grid < 1) grid = 1;
  const cudaError_t err = launch_tc_any<NB>(L, *bt, grid, st);
  delete bt;
  return (int)err;
}

int launch_tc_single(const TcLaunch &L, const TcWork *works, const int2 *glist, const int *glist_n, cudaStream_t st);

int launch_tc(const TcLaunch &L, const TcWork *works, int n, const int2 *glist, const int *glist_n, cudaStream_t st) {
  if (n == 1) return launch_tc_single(L, works, glist, glist_n, st);
  return launch_tc_nb<TC_MAXB>(L, works, n, glist, glist_n, st);
}

}  // namespace dotpe
