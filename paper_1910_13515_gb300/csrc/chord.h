// chord.h -- launcher of the FP64 step kernels with the chord-Newton hybrid
// root finder (chord.cu).
#pragma once
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace lbm39 {

// One step pass (even or odd AA pass) of every fluid cell, FP64, solving the
// constraint equations with newton_chord; false on a launch error.
bool launch_step_chord(const Desc& d, bool odd, cudaStream_t stream);

}  // namespace lbm39
