// prandtl.cu -- the step kernels with the Prandtl-number adjustment
// (lbm39_params.prandtl != 1): the same fused step as the paper's Pr = 1
// collision, with the quasi-equilibrium correction of g (kernels.cuh,
// relax_push<..., PR = true>), instantiated in a translation unit of their own
// so that the Pr = 1 kernels carry none of it and the library compiles in
// parallel.  These lattices always solve all 13 constraints (no z-mirror
// reduction).
#include <cuda_runtime.h>

#include "kernels.cuh"
#include "prandtl.h"

namespace lbm39 {

namespace {
constexpr int BLK = 64;  // the step kernel's block (the workspace is laid out per block)
constexpr size_t WS_BYTES = (size_t)BLK * WS_DOUBLES * sizeof(double);
}  // namespace

bool launch_step_prandtl(const Desc& d, bool odd, bool mixed, cudaStream_t stream) {
  const unsigned grid = (unsigned)((d.N + BLK - 1) / BLK);
  if (mixed) {
    if (odd) k_step<true, float, BLK, false, true><<<grid, BLK, WS_BYTES, stream>>>(d);
    else k_step<false, float, BLK, false, true><<<grid, BLK, WS_BYTES, stream>>>(d);
  } else {
    if (odd) k_step<true, double, BLK, false, true><<<grid, BLK, WS_BYTES, stream>>>(d);
    else k_step<false, double, BLK, false, true><<<grid, BLK, WS_BYTES, stream>>>(d);
  }
  return cudaGetLastError() == cudaSuccess;
}

}  // namespace lbm39
