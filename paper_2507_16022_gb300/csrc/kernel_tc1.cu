// The fused tcgen05 kernel instantiated for one event per launch (its own
// translation unit so that the two instantiation sets compile in parallel).
#include "kernel_tc.cuh"

namespace dotpe {

int launch_tc_single(const TcLaunch &L, const TcWork *works, const int2 *glist, const int *glist_n, cudaStream_t st) {
  const int tev = L.tev == 64 ? 64 : 32;
  TcBatch<1> bt;
  bt.w[0] = works[0];
  bt.mapB[0] = (tev == 64) ? works[0].mapB64 : works[0].mapB;
  bt.begin[0] = 0;
  bt.begin[1] = tc_work_items(works[0], tev);
  bt.n = 1;
  bt.glist = glist;
  bt.glist_n = glist_n;
  bt.gate = L.gate;
  bt.gate_want = L.gate_want;
  const int total = bt.begin[1];
  int grid = (glist || L.n_sms < total) ? L.n_sms : total;
  if (grid < 1) grid = 1;
  const cudaError_t err = launch_tc_any<1>(L, bt, grid, st);
  return (int)err;
}

}  // namespace dotpe
