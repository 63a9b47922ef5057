// chord.cu -- the FP64 step kernels with the chord-Newton hybrid root finder
// (lbm39_params.root_finder = 1; cell.cuh newton_chord): the same fused step
// with another solver of the 13 (or, z-mirror reduced, 9) constraint
// equations, instantiated in a translation unit of its own so that the
// Newton kernels are untouched and the library compiles in parallel.
#include <cuda_runtime.h>

#include "chord.h"
#include "kernels.cuh"

namespace lbm39 {

namespace {
constexpr int BLK = 64;  // the step kernel's block (the workspace is laid out per block)
constexpr size_t WS_BYTES = (size_t)BLK * WS_DOUBLES * sizeof(double);
}  // namespace

bool launch_step_chord(const Desc& d, bool odd, cudaStream_t stream) {
  const unsigned grid = (unsigned)((d.N + BLK - 1) / BLK);
  if (d.d2) {
    if (odd) k_step<true, double, BLK, true, false, true><<<grid, BLK, WS_BYTES, stream>>>(d);
    else k_step<false, double, BLK, true, false, true><<<grid, BLK, WS_BYTES, stream>>>(d);
  } else {
    if (odd) k_step<true, double, BLK, false, false, true><<<grid, BLK, WS_BYTES, stream>>>(d);
    else k_step<false, double, BLK, false, false, true><<<grid, BLK, WS_BYTES, stream>>>(d);
  }
  return cudaGetLastError() == cudaSuccess;
}

}  // namespace lbm39
