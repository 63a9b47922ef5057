// root_finders.h -- launcher of the FP64 step kernels with the other root
// finders of the constraint equations (root_finders.cu).
#pragma once
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace lbm39 {

// One step pass (even or odd AA pass) of every fluid cell, FP64, solving the
// constraint equations with root finder `solver` (1: chord-Newton hybrid,
// 2: Newton with a single-precision direction); false on a launch error or
// another solver.
bool launch_step_root_finder(const Desc& d, bool odd, int solver, cudaStream_t stream);

}  // namespace lbm39
