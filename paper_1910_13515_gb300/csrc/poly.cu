// poly.cu -- the paper's comparison model (Sec. 5) on the GPU: D3Q39
// double-distribution BGK with the fourth-order polynomial equilibrium of
// poly_eq.cuh, for periodic lattices, on the in-place AA pattern and the
// generated moment sums of the 13-moment step (kernels.cuh); and its C ABI
// (include/lbm39_poly.h).
//
// One kernel per AA pass: each thread takes one cell, gathers f and g, forms
// rho, u, T, then for each (xi, -xi) pair the scaled equilibrium values and
// the post-collision populations, pushed straight away.  No per-cell state
// besides the 78 populations.
#include <cuda_runtime.h>

#include <new>

#include "../../include/lbm39.h"
#include "../../include/lbm39_poly.h"
#include "kernels.cuh"
#include "poly_eq.cuh"

namespace lbm39 {
namespace poly {

constexpr int BLK = 128;          // threads per block of the cell kernels
constexpr int RED_BLOCKS = 1024;  // blocks of the conserved-sum reduction
constexpr int RED_THREADS = 128;

// Pre-collision population i of one distribution (base 0: f, Q: g) of the
// cell at the lattice's current time (the AA rule of gather()).
template <bool ODD, int i>
__device__ __forceinline__ double load_pre(const Desc& d, long long cell, const Nbr& nb,
                                           int base) {
  const double* __restrict__ pop = static_cast<const double*>(d.pop);
  if constexpr (!ODD) {
    return pop[(long long)(base + i) * d.Np + cell];
  } else {
    constexpr int cx = CX[i], cy = CY[i], cz = CZ[i];
    return pop[(long long)(base + opp(i)) * d.Np + nb.at(-cx, -cy, -cz)];
  }
}

// One cell's step.  With omega = 1/tau and W_i = omega rho w_i,
// omega f_i^eq = W_i P_i (pair_values), h* = (1 - omega) h + omega h^eq and
// omega g_i^eq = (2 C_v - D) T omega f_i^eq.  Both members of a pair are read
// before either is written: in place, the even pass writes h*_i into slot
// opp(i) and the odd pass writes over the slot read for opp(i).
template <bool ODD>
__device__ __forceinline__ void step_cell(const Desc& d, long long cell) {
  Nbr nb;
  if constexpr (ODD) nb = Nbr(d, coord_of(d, cell));
  double f[Q];
  gather<ODD, double>(d, cell, nb, 0, f);
  double rho, jx, jy, jz, e2;
  gen::f_moments<double>(f, rho, jx, jy, jz, e2);
  {
    double g[Q];
    gather<ODD, double>(d, cell, nb, Q, g);
    e2 += gen::g_sum<double>(g);
  }
  const Macro M = macro_from_moments(rho, jx, jy, jz, e2, d.ph.inv_2cv);
  const Coef k = coefficients(M.ux * M.ux + M.uy * M.uy + M.uz * M.uz, M.T - TH);
  const double om = d.ph.omega[0];
  const double keep = 1.0 - om;
  const double scale = om * rho;
  const double cgT = d.ph.cg * M.T;
  {
    const double q0 = scale * weight(0) * k.a00;
    const double g0 = load_pre<ODD, 0>(d, cell, nb, Q);
    push<ODD, double, 0>(d, cell, nb, 0, fma(keep, f[0], q0));
    push<ODD, double, 0>(d, cell, nb, Q, fma(keep, g0, cgT * q0));
  }
  pairs_for<0, (Q - 1) / 2>([&](auto P) {
    constexpr int i = decltype(P)::value, j = i + 1;
    double qp, qm;
    pair_values<i>(k, scale, M.ux, M.uy, M.uz, qp, qm);
    const double gi = load_pre<ODD, i>(d, cell, nb, Q);
    const double gj = load_pre<ODD, j>(d, cell, nb, Q);
    push<ODD, double, i>(d, cell, nb, 0, fma(keep, f[i], qp));
    push<ODD, double, j>(d, cell, nb, 0, fma(keep, f[j], qm));
    push<ODD, double, i>(d, cell, nb, Q, fma(keep, gi, cgT * qp));
    push<ODD, double, j>(d, cell, nb, Q, fma(keep, gj, cgT * qm));
  });
}

template <bool ODD>
__global__ void __launch_bounds__(BLK) k_poly_step(Desc d) {
  const long long cell = (long long)blockIdx.x * BLK + threadIdx.x;
  if (cell < d.N) step_cell<ODD>(d, cell);
}

// f = f^eq, g = g^eq at even time (own slots).
__global__ void __launch_bounds__(BLK) k_poly_init(Desc d, const double* rho, const double* u,
                                                   const double* T) {
  const long long cell = (long long)blockIdx.x * BLK + threadIdx.x;
  if (cell >= d.N) return;
  double* __restrict__ pop = static_cast<double*>(d.pop);
  double fe[Q];
  const double Tc = T[cell];
  feq_cell(rho[cell], u[cell], u[d.N + cell], u[2 * d.N + cell], Tc, fe);
  const double cgT = d.ph.cg * Tc;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    pop[(long long)i * d.Np + cell] = fe[i];
    pop[(long long)(Q + i) * d.Np + cell] = cgT * fe[i];
  }
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
long long plane_stride(long long N) { return (N + 63) / 64 * 64; }

struct AuxLayout {
  size_t partials, result, total;
};

AuxLayout aux_layout() {
  AuxLayout a;
  size_t off = 0;
  a.partials = off; off = align256(off + sizeof(double) * 5 * RED_BLOCKS);
  a.result = off; off = align256(off + sizeof(double) * 8);
  a.total = off;
  return a;
}

bool params_ok(const lbm39_params* p) {
  if (!p) return false;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return false;
  const long long N = (long long)p->nx * p->ny * p->nz;
  if (N > (1LL << 31) - 64) return false;
  if (!(p->gamma > 1.0) || !(p->tau >= 0.5)) return false;
  if (p->precision != LBM39_FP64 || p->kn_sensor != 0) return false;
  return p->periodic[0] && p->periodic[1] && p->periodic[2];
}

}  // namespace poly
}  // namespace lbm39

using namespace lbm39;

struct lbm39_poly {
  lbm39_params p;
  long long N = 0, Np = 0;
  char* aux = nullptr;
  poly::AuxLayout lay{};
  cudaStream_t stream = nullptr;
  long long t = 0;
  bool initialized = false;
  Desc desc{};
};

static int launched() { return cudaGetLastError() == cudaSuccess ? LBM39_OK : LBM39_ERR_CUDA; }

extern "C" {

int lbm39_poly_query_bytes(const lbm39_params* p, size_t* pop_bytes, size_t* aux_bytes) {
  if (!poly::params_ok(p) || !pop_bytes || !aux_bytes) return LBM39_ERR_ARG;
  const long long N = (long long)p->nx * p->ny * p->nz;
  *pop_bytes = sizeof(double) * 2 * Q * (size_t)poly::plane_stride(N);
  *aux_bytes = poly::aux_layout().total;
  return LBM39_OK;
}

int lbm39_poly_create(const lbm39_params* p, void* pop_buf, void* aux_buf, void* cuda_stream,
                      lbm39_poly** out) {
  if (!out) return LBM39_ERR_ARG;
  *out = nullptr;
  if (!poly::params_ok(p) || !pop_buf || !aux_buf) return LBM39_ERR_ARG;
  if (((uintptr_t)pop_buf & 255) || ((uintptr_t)aux_buf & 255)) return LBM39_ERR_ARG;
  lbm39_poly* L = new (std::nothrow) lbm39_poly;
  if (!L) return LBM39_ERR_ARG;
  L->p = *p;
  L->N = (long long)p->nx * p->ny * p->nz;
  L->Np = poly::plane_stride(L->N);
  L->aux = static_cast<char*>(aux_buf);
  L->lay = poly::aux_layout();
  L->stream = static_cast<cudaStream_t>(cuda_stream);
  Desc& d = L->desc;
  d.pop = pop_buf;
  d.N = L->N;
  d.Np = L->Np;
  d.nx = p->nx; d.ny = p->ny; d.nz = p->nz;
  for (int a = 0; a < 3; ++a) d.per[a] = 1;
  const double cv = 1.0 / (p->gamma - 1.0);
  d.ph.tau = p->tau;
  d.ph.cg = 2.0 * cv - D;
  d.ph.inv_2cv = 1.0 / (2.0 * cv);
  for (int b = 0; b < 4; ++b) d.ph.omega[b] = 1.0 / p->tau;
  *out = L;
  return LBM39_OK;
}

int lbm39_poly_init(lbm39_poly* L, const double* rho, const double* u, const double* T) {
  if (!L || !rho || !u || !T) return LBM39_ERR_ARG;
  const unsigned grid = (unsigned)((L->N + poly::BLK - 1) / poly::BLK);
  poly::k_poly_init<<<grid, poly::BLK, 0, L->stream>>>(L->desc, rho, u, T);
  if (launched() != LBM39_OK) return LBM39_ERR_CUDA;
  L->t = 0;
  L->initialized = true;
  return LBM39_OK;
}

int lbm39_poly_step(lbm39_poly* L, int64_t nsteps) {
  if (!L || nsteps < 0) return LBM39_ERR_ARG;
  if (!L->initialized) return LBM39_ERR_STATE;
  const unsigned grid = (unsigned)((L->N + poly::BLK - 1) / poly::BLK);
  for (int64_t s = 0; s < nsteps; ++s) {
    if (L->t & 1) poly::k_poly_step<true><<<grid, poly::BLK, 0, L->stream>>>(L->desc);
    else poly::k_poly_step<false><<<grid, poly::BLK, 0, L->stream>>>(L->desc);
    if (launched() != LBM39_OK) return LBM39_ERR_CUDA;
    ++L->t;
  }
  return LBM39_OK;
}

int lbm39_poly_read(lbm39_poly* L, double* rho, double* u, double* T, double* p) {
  if (!L) return LBM39_ERR_ARG;
  if (!L->initialized) return LBM39_ERR_STATE;
  const unsigned grid = (unsigned)((L->N + 127) / 128);
  if (L->t & 1)
    k_macros<true, double><<<grid, 128, 0, L->stream>>>(L->desc, rho, u, L->N, T, p, 0, L->N);
  else
    k_macros<false, double><<<grid, 128, 0, L->stream>>>(L->desc, rho, u, L->N, T, p, 0, L->N);
  return launched();
}

int lbm39_poly_conserved(lbm39_poly* L, double* sums5) {
  if (!L || !sums5) return LBM39_ERR_ARG;
  if (!L->initialized) return LBM39_ERR_STATE;
  double* partials = reinterpret_cast<double*>(L->aux + L->lay.partials);
  double* result = reinterpret_cast<double*>(L->aux + L->lay.result);
  if (L->t & 1)
    k_conserved<true, double, poly::RED_THREADS>
        <<<poly::RED_BLOCKS, poly::RED_THREADS, 0, L->stream>>>(L->desc, partials);
  else
    k_conserved<false, double, poly::RED_THREADS>
        <<<poly::RED_BLOCKS, poly::RED_THREADS, 0, L->stream>>>(L->desc, partials);
  k_sum_partials<<<1, 32, 0, L->stream>>>(partials, poly::RED_BLOCKS, result);
  if (launched() != LBM39_OK) return LBM39_ERR_CUDA;
  if (cudaMemcpyAsync(sums5, result, 5 * sizeof(double), cudaMemcpyDeviceToHost, L->stream) !=
      cudaSuccess)
    return LBM39_ERR_CUDA;
  return cudaStreamSynchronize(L->stream) == cudaSuccess ? LBM39_OK : LBM39_ERR_CUDA;
}

int64_t lbm39_poly_time(const lbm39_poly* L) { return L ? L->t : -1; }

void lbm39_poly_destroy(lbm39_poly* L) { delete L; }

}  // extern "C"
