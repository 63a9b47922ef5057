// batch.cuh -- kernels of the serving form: many resident lattices advanced
// by one packed launch per time step.  A tile is one block of one lattice;
// each lattice keeps its own time (and therefore its own AA parity) and stops
// at its own end time, so a packed run gives every lattice exactly the
// arithmetic of stepping it alone.
#pragma once

#include "kernels.cuh"

namespace lbm39 {

struct BatchEntry {
  Desc d;
  long long t0;     // the lattice's time at step index 0 of the current launch sequence
  long long t_end;  // the lattice does not step past this time
};

struct Tile {
  int lat;          // index into the batch entries
  int pad;
  long long cell0;  // first cell of the tile
};

// D2: every lattice of these tiles takes the nine-constraint (z-mirror) solve
// (FP64 lattices one cell thick in z with u_z = 0); the host sorts the tiles by
// constraint system and launches one instantiation for each.
template <class P, int BLK, bool D2>
__global__ void __launch_bounds__(BLK) k_batch_step(const BatchEntry* __restrict__ E,
                                                    const Tile* __restrict__ tiles, int s) {
  extern __shared__ double smem[];
  __shared__ unsigned int s_ctr[CTR_N];
  __shared__ Desc sd;
  __shared__ long long st;
  const Tile tl = tiles[blockIdx.x];
  if (threadIdx.x == 0) {
    sd = E[tl.lat].d;
    st = E[tl.lat].t0 + s < E[tl.lat].t_end ? E[tl.lat].t0 + s : -1;
    sd.t = st;
  }
  for (int k = threadIdx.x; k < CTR_N; k += BLK) s_ctr[k] = 0;
  load_exp_table();  // also publishes sd and st
  const long long t = st;
  if (t < 0) return;  // this lattice has reached its end time (uniform over the block)
  const long long cell = tl.cell0 + threadIdx.x;
  if (cell < sd.N && (sd.mask == nullptr || sd.mask[cell] == MASK_FLUID)) {
    WS<BLK> w{smem + threadIdx.x};
    if (t & 1) step_cell<true, P, BLK, D2>(sd, cell, w, s_ctr);
    else step_cell<false, P, BLK, D2>(sd, cell, w, s_ctr);
  }
  flush_stats<BLK>(s_ctr, sd.ctr);
}

// Boundary fills of the lattices that have freestream or outflow cells.
template <class P>
__global__ void k_batch_fill(const BatchEntry* __restrict__ E, const Tile* __restrict__ tiles,
                             int s) {
  const Tile tl = tiles[blockIdx.x];
  const BatchEntry& e = E[tl.lat];
  const long long t = e.t0 + s;
  if (t >= e.t_end) return;
  const long long cell = tl.cell0 + threadIdx.x;
  if (cell >= e.d.N) return;
  if (t & 1) fill_odd_cell<P>(e.d, cell);
  else fill_even_cell<P>(e.d, cell);
}

// After a launch sequence of n steps: every lattice's t0 moves on by n.
__global__ void k_batch_advance(BatchEntry* E, int nlat, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nlat) E[j].t0 += n;
}

}  // namespace lbm39
