// The fused tcgen05 kernel instantiated for one event per launch (its own
// translation unit so that the two instantiation sets compile in parallel).
#include "kernel_tc.cuh"

namespace dotpe {

int launch_tc_single(const TcLaunch &L, const TcWork *works, const int2 *glist, const int *glist_n, cudaStream_t st) {
  TcBatch<1> bt;
  bt.w[0] = works[0];
  bt.mapB[0] = works[0].mapB;
  bt.begin[0] = 0;
  bt.begin[1] = works[0].n_itile * works[0].n_etile;
  bt.n = 1;
  bt.glist = glist;
  bt.glist_n = glist_n;
  const int total = bt.begin[1];
  int grid = (glist || L.n_sms < total) ? L.n_sms : total;
  if (grid < 1) grid = 1;
  auto go = [&](auto kern, size_t smem) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, NT, smem, st>>>(L.mapA, bt, L.C);
    return cudaGetLastError();
  };
  cudaError_t err;
  if (L.split && L.bf16) {
    err = L.consec ? go(tc_fused_kernel<true, true, true, 1>, smem_bytes<true>())
                   : go(tc_fused_kernel<true, false, true, 1>, smem_bytes<true>());
  } else if (L.split) {
    err = L.consec ? go(tc_fused_kernel<false, true, true, 1>, smem_bytes<true>())
                   : go(tc_fused_kernel<false, false, true, 1>, smem_bytes<true>());
  } else if (L.bf16) {
    err = L.consec ? go(tc_fused_kernel<true, true, false, 1>, smem_bytes<false>())
                   : go(tc_fused_kernel<true, false, false, 1>, smem_bytes<false>());
  } else {
    err = L.consec ? go(tc_fused_kernel<false, true, false, 1>, smem_bytes<false>())
                   : go(tc_fused_kernel<false, false, false, 1>, smem_bytes<false>());
  }
  return (int)err;
}

}  // namespace dotpe
