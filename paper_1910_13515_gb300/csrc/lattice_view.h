// lattice_view.h -- what the library's other translation units (diag.cu) may
// read of a 13-moment lattice handle, defined in lbm39.cu.
#pragma once
#include <cuda_runtime.h>

#include "kernels.cuh"

struct lbm39_lattice;

namespace lbm39 {

struct LatticeView {
  Desc desc;            // the kernels' descriptor, its time set to the lattice's time
  cudaStream_t stream;  // the lattice's stream
  long long N;          // cells
  bool mixed;           // precision form (FP32 deviation storage)
  bool initialized;     // lbm39_init has run
  int solver;           // root finder of the FP64 path (lbm39_params.root_finder)
};

// False for a NULL lattice or view.
bool lattice_view(const lbm39_lattice* L, LatticeView* v);

}  // namespace lbm39
