// root_finders.cu -- the FP64 step kernels with the other root finders of the
// constraint equations (lbm39_params.root_finder): 1, the chord-Newton hybrid
// (cell.cuh newton_chord); 2, Newton with a single-precision direction
// (cell.cuh newton<BLK, true>); 3, that after a single-precision start
// (cell.cuh start32).  The same fused step with another solver,
// instantiated in a translation unit of its own so that the Newton kernels are
// untouched and the library compiles in parallel.
#include <cuda_runtime.h>

#include "kernels.cuh"
#include "root_finders.h"

namespace lbm39 {

namespace {
constexpr int BLK = 64;  // the step kernel's block (the workspace is laid out per block)
constexpr size_t WS_BYTES = (size_t)BLK * WS_DOUBLES * sizeof(double);

template <int SOLVER>
void launch(const Desc& d, bool odd, cudaStream_t stream, unsigned grid) {
  if (d.d2) {
    if (odd) k_step<true, double, BLK, true, false, SOLVER><<<grid, BLK, WS_BYTES, stream>>>(d);
    else k_step<false, double, BLK, true, false, SOLVER><<<grid, BLK, WS_BYTES, stream>>>(d);
  } else {
    if (odd) k_step<true, double, BLK, false, false, SOLVER><<<grid, BLK, WS_BYTES, stream>>>(d);
    else k_step<false, double, BLK, false, false, SOLVER><<<grid, BLK, WS_BYTES, stream>>>(d);
  }
}
}  // namespace

bool launch_step_root_finder(const Desc& d, bool odd, int solver, cudaStream_t stream) {
  const unsigned grid = (unsigned)((d.N + BLK - 1) / BLK);
  if (solver == 1) launch<1>(d, odd, stream, grid);
  else if (solver == 2) launch<2>(d, odd, stream, grid);
  else if (solver == 3) launch<3>(d, odd, stream, grid);
  else return false;
  return cudaGetLastError() == cudaSuccess;
}

}  // namespace lbm39
