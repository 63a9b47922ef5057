// prandtl.h -- launcher of the Prandtl-adjusted step kernels (prandtl.cu).
#pragma once
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace lbm39 {

// One step pass (even or odd AA pass) of every fluid cell with the
// Prandtl-number adjustment, FP64 or precision form; false on a launch error.
bool launch_step_prandtl(const Desc& d, bool odd, bool mixed, cudaStream_t stream);

}  // namespace lbm39
