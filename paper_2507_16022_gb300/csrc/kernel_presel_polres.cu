// The tensor-core pre-selection kernel instantiated for a polarisation-resolved bank
// (its own translation unit, so that the instantiation sets compile in parallel).
#include "kernel_presel.cuh"

namespace dotpe {

template <int VAR>
cudaError_t launch_presel_var(const CUtensorMap &mapG, const CUtensorMap &mapBank, const PreselParams &p, bool bf16,
                              bool split, int grid, cudaStream_t st);
template <>
cudaError_t launch_presel_var<2>(const CUtensorMap &mapG, const CUtensorMap &mapBank, const PreselParams &p,
                                 bool bf16, bool split, int grid, cudaStream_t st) {
  return launch_presel_pm<2>(mapG, mapBank, p, bf16, split, grid, st);
}

}  // namespace dotpe
