// diag.cu -- per-cell diagnostic fields of a 13-moment lattice's current state:
// the Knudsen sensor eps (Eq. DeltaAvg) and the number of Newton updates the
// next step's solve takes, the two quantities the paper maps over the airfoil
// flow (Sec. 4).  Each cell does the next step's work up to its collision
// (moments, targets, the warm-started solve from the stored multipliers with
// the same retry schedule and root finder, the fallback equilibrium where the
// solve fails) and
// writes the two values; no population, multiplier or counter changes.
#include <cuda_runtime.h>

#include "../../include/lbm39.h"
#include "kernels.cuh"
#include "lattice_view.h"

namespace lbm39 {
namespace {

constexpr int BLK = 64;  // the step kernel's block (the workspace is laid out per block)
constexpr size_t WS_BYTES = (size_t)BLK * WS_DOUBLES * sizeof(double);

// f_i of the current state in FP64 (the stored deviation plus h_ref in the
// precision form; exact).
template <bool ODD, class P>
__device__ __forceinline__ void gather_f(const Desc& d, long long cell, double (&f)[Q]) {
  Nbr nb;
  if constexpr (ODD) nb = Nbr(d, coord_of(d, cell));
  P h[Q];
  gather<ODD, P>(d, cell, nb, 0, h);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if constexpr (sizeof(P) == 8) f[i] = h[i];
    else f[i] = (double)h[i] + d.href[i];
  }
}

template <class P>
__device__ __forceinline__ Macro moments_at(const Desc& d, long long cell, bool odd) {
  Nbr nb;
  if (odd) {
    nb = Nbr(d, coord_of(d, cell));
    return gather_moments<true, P>(d, cell, nb);
  }
  return gather_moments<false, P>(d, cell, nb);
}

// eps: FP64 (1/Q) sum_i |f_i - f_i^eq| / f_i^eq of the state against the
// equilibrium the next step relaxes to; n_upd: its Newton updates, -1 where
// the solve fails (the cell takes the fallback equilibrium).  Non-fluid cells
// read 0.  odd: the AA parity of the lattice's time.
template <class P, bool D2, int SOLVER = 0>
__global__ void __launch_bounds__(BLK) k_diag_fields(Desc d, int odd, double* eps_out,
                                                     int* nupd_out) {
  extern __shared__ double smem[];
  load_exp_table();
  const long long cell = (long long)blockIdx.x * BLK + threadIdx.x;
  if (cell >= d.N) return;
  if (d.mask != nullptr && d.mask[cell] != MASK_FLUID) {
    eps_out[cell] = 0.0;
    nupd_out[cell] = 0;
    return;
  }
  WS<BLK> w{smem + threadIdx.x};
  WS<BLK> F = w.at(WS_E), lam = w.at(WS_LAM), m = w.at(WS_M);
  const Macro M = moments_at<P>(d, cell, odd != 0);
  targets<BLK>(M.ux, M.uy, M.uz, M.T, m);
  load_solver_state<BLK>(d, cell, w);
  const bool marked = is_fallback_embedding<BLK>(lam);
  const int maxit = !marked ? d.ph.maxit : retry_budget(d.t, d.ph.maxit);
  int n32;
  const NewtonResult nr = solve_cell<P, BLK, D2, SOLVER>(w, d.ph, maxit, n32);
  if (nr.failed) fallback_cell<BLK>(d.lam, d.Np, cell, w, M.T, marked);
  double f[Q];
  if (odd) gather_f<true, P>(d, cell, f);
  else gather_f<false, P>(d, cell, f);
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const double feq = M.rho * F[i];
    s += fabs(f[i] - feq) / feq;
  }
  eps_out[cell] = s * (1.0 / Q);
  nupd_out[cell] = nr.failed ? -1 : nr.n_upd;
}

}  // namespace
}  // namespace lbm39

extern "C" int lbm39_diag_fields(lbm39_lattice* L, double* eps, int32_t* n_upd) {
  using namespace lbm39;
  LatticeView v;
  if (!lattice_view(L, &v) || !eps || !n_upd) return LBM39_ERR_ARG;
  if (!v.initialized) return LBM39_ERR_STATE;
  const unsigned grid = (unsigned)((v.N + BLK - 1) / BLK);
  const int odd = (int)(v.desc.t & 1);
  if (v.mixed)
    k_diag_fields<float, false><<<grid, BLK, WS_BYTES, v.stream>>>(v.desc, odd, eps, n_upd);
  else if (v.solver == 1 && v.desc.d2)
    k_diag_fields<double, true, 1><<<grid, BLK, WS_BYTES, v.stream>>>(v.desc, odd, eps, n_upd);
  else if (v.solver == 1)
    k_diag_fields<double, false, 1><<<grid, BLK, WS_BYTES, v.stream>>>(v.desc, odd, eps, n_upd);
  else if (v.solver == 2 && v.desc.d2)
    k_diag_fields<double, true, 2><<<grid, BLK, WS_BYTES, v.stream>>>(v.desc, odd, eps, n_upd);
  else if (v.solver == 2)
    k_diag_fields<double, false, 2><<<grid, BLK, WS_BYTES, v.stream>>>(v.desc, odd, eps, n_upd);
  else if (v.solver == 3 && v.desc.d2)
    k_diag_fields<double, true, 3><<<grid, BLK, WS_BYTES, v.stream>>>(v.desc, odd, eps, n_upd);
  else if (v.solver == 3)
    k_diag_fields<double, false, 3><<<grid, BLK, WS_BYTES, v.stream>>>(v.desc, odd, eps, n_upd);
  else if (v.desc.d2)
    k_diag_fields<double, true><<<grid, BLK, WS_BYTES, v.stream>>>(v.desc, odd, eps, n_upd);
  else
    k_diag_fields<double, false><<<grid, BLK, WS_BYTES, v.stream>>>(v.desc, odd, eps, n_upd);
  return cudaGetLastError() == cudaSuccess ? LBM39_OK : LBM39_ERR_CUDA;
}
