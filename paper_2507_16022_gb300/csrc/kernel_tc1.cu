// The fused tcgen05 kernel instantiated for one event per launch (its own
// translation unit so that the two instantiation sets compile in parallel).
#include <algorithm>

#include "kernel_tc.cuh"

namespace dotpe {

int launch_tc_single(const TcLaunch &L, const TcWork *works, const int2 *glist, const int *glist_n, cudaStream_t st) {
  const int tev = L.tev == 64 ? 64 : 32;
  // CTA pairs: 64-sample tiles in grid order; each CTA loads half of the tile's
  // extrinsic rows, so through the 64-row boxes of the 32-sample map
  const bool pair = L.pair && tev == 64 && !glist && !L.split && !L.pol;
  TcLaunch Lp = L;
  Lp.pair = pair;
  TcBatch<1> bt;
  bt.w[0] = works[0];
  bt.mapB[0] = (tev == 64 && !pair) ? works[0].mapB64 : works[0].mapB;
  bt.begin[0] = 0;
  bt.begin[1] = tc_work_items(works[0], tev, pair);
  bt.n = 1;
  bt.glist = glist;
  bt.glist_n = glist_n;
  bt.gate = L.gate;
  bt.gate_want = L.gate_want;
  const int total = bt.begin[1];
  int grid = (glist || L.n_sms < total) ? L.n_sms : total;
  if (grid < 1) grid = 1;
  if (pair) grid = 2 * std::max(1, std::min(L.n_sms / 2, total));  // one cluster per pair tile at most
  const cudaError_t err = launch_tc_any<1>(Lp, bt, grid, st);
  return (int)err;
}

}  // namespace dotpe
