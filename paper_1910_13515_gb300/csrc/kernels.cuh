// kernels.cuh -- CUDA kernels of the D3Q39 DDF step: initial equilibrium, the
// fused collide-and-stream passes (AA pattern), boundary fills, macroscopic
// read-out and conserved sums.
//
// Storage: 78 planes of Np elements (f_0..f_38 then g_0..g_38), x fastest.
// AA pattern over one buffer.  At even time the buffer holds the
// pre-collision populations h_i(x) in slot (x, i).  The even pass reads its
// own slots, collides and writes h*_i(x) into slot (x, opp i).  The odd pass
// gathers h_i(x) = h*_i(x - xi_i) from slot (x - xi_i, opp i), collides and
// pushes h*_i(x) into slot (x + xi_i, i), which is the pre-collision h_i of
// the next time step.  Every slot is read and written by one thread only.
// Half-way bounce-back: a source (odd gather) or destination (odd push) that
// is solid redirects to the cell's own slot of the opposite direction.
// Freestream and outflow cells never collide; the fill kernels give the
// fluid cells what those cells would have streamed (Sec. 4 boundary kinds).
#pragma once
#include <cstdint>

#include "cell.cuh"

namespace lbm39 {

struct Desc {
  double* pop;                 // 78 planes
  double* lam;                 // 13 planes, multipliers kept between steps
  const uint8_t* mask;         // nullptr: every cell fluid, all axes periodic
  unsigned long long* ctr;     // counters (see CTR_*)
  const double* heq_inf;       // 78 far-field equilibrium populations
  long long N, Np;             // cells, plane stride in elements
  int nx, ny, nz;
  int per[3];                  // periodic axes
  Phys ph;
};

enum { CTR_FAILED = 0, CTR_UPDATES = 1, CTR_HIST = 2, CTR_EPS = 34, CTR_N = 38 };

struct Coord {
  int x, y, z;
};

__device__ __forceinline__ Coord coord_of(const Desc& d, long long cell) {
  const long long yz = cell / d.nx;
  return Coord{int(cell - yz * d.nx), int(yz % d.ny), int(yz / d.ny)};
}

__device__ __forceinline__ int wrap(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

// Index of the cell at x + (dx, dy, dz) with periodic wrap of every axis
// (non-periodic axes carry boundary layers, so fluid cells never wrap there).
struct Nbr {
  int xs[7];
  long long ys[7], zs[7];
  __device__ __forceinline__ Nbr(const Desc& d, Coord c) {
#pragma unroll
    for (int s = 0; s < 7; ++s) {
      xs[s] = wrap(c.x + s - 3, d.nx);
      ys[s] = (long long)wrap(c.y + s - 3, d.ny) * d.nx;
      zs[s] = (long long)wrap(c.z + s - 3, d.nz) * d.nx * d.ny;
    }
  }
  __device__ __forceinline__ long long at(int dx, int dy, int dz) const {
    return xs[dx + 3] + ys[dy + 3] + zs[dz + 3];
  }
};

// Pre-collision populations of fluid cell `cell` at the lattice's current time:
// own slots at even time, the odd gather (with bounce-back) at odd time.
template <bool ODD, int BLK>
__device__ __forceinline__ void gather(const Desc& d, long long cell, WS<BLK> w) {
  const double* __restrict__ P = d.pop;
  if constexpr (!ODD) {
    static_for<0, 2 * Q>([&](auto I) {
      constexpr int j = decltype(I)::value;
      w[j] = P[j * d.Np + cell];
    });
  } else {
    const Nbr nb(d, coord_of(d, cell));
    static_for<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      constexpr int cx = CX[i], cy = CY[i], cz = CZ[i];
      const long long s = nb.at(-cx, -cy, -cz);
      const bool solid = d.mask != nullptr && d.mask[s] == MASK_SOLID;
      const long long src = solid ? (long long)i * d.Np + cell : (long long)opp(i) * d.Np + s;
      w[WS_F + i] = P[src];
      w[WS_G + i] = P[src + Q * d.Np];
    });
  }
}

// Post-collision populations of fluid cell `cell` into their AA slots.
template <bool ODD, int BLK>
__device__ __forceinline__ void scatter(const Desc& d, long long cell, WS<BLK> w) {
  double* __restrict__ P = d.pop;
  if constexpr (!ODD) {
    static_for<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      P[(long long)opp(i) * d.Np + cell] = w[WS_F + i];
      P[(long long)(Q + opp(i)) * d.Np + cell] = w[WS_G + i];
    });
  } else {
    const Nbr nb(d, coord_of(d, cell));
    static_for<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      constexpr int cx = CX[i], cy = CY[i], cz = CZ[i];
      const long long t = nb.at(cx, cy, cz);
      const bool solid = d.mask != nullptr && d.mask[t] == MASK_SOLID;
      const long long dst = solid ? (long long)opp(i) * d.Np + cell : (long long)i * d.Np + t;
      P[dst] = w[WS_F + i];
      P[dst + Q * d.Np] = w[WS_G + i];
    });
  }
}

template <int BLK>
__device__ __forceinline__ void flush_stats(unsigned int* s_ctr, unsigned long long* ctr) {
  __syncthreads();
  for (int k = threadIdx.x; k < CTR_N; k += BLK)
    if (s_ctr[k]) atomicAdd(ctr + k, (unsigned long long)s_ctr[k]);
}

// One time step over every fluid cell (even or odd AA pass).
template <bool ODD, int BLK>
__global__ void __launch_bounds__(BLK) k_step(Desc d) {
  extern __shared__ double smem[];
  __shared__ unsigned int s_ctr[CTR_N];
  for (int k = threadIdx.x; k < CTR_N; k += BLK) s_ctr[k] = 0;
  __syncthreads();
  const long long cell = (long long)blockIdx.x * BLK + threadIdx.x;
  const bool active =
      cell < d.N && (d.mask == nullptr || d.mask[cell] == MASK_FLUID);
  if (active) {
    WS<BLK> w{smem + threadIdx.x};
    gather<ODD, BLK>(d, cell, w);
#pragma unroll
    for (int k = 0; k < NM; ++k) w[WS_LAM + k] = d.lam[k * d.Np + cell];
    const CellStats cs = collide_fp64<BLK>(w, d.ph);
#pragma unroll
    for (int k = 0; k < NM; ++k) d.lam[k * d.Np + cell] = w[WS_LAM + k];
    scatter<ODD, BLK>(d, cell, w);
    atomicAdd(&s_ctr[CTR_FAILED], (unsigned)cs.failed);
    atomicAdd(&s_ctr[CTR_UPDATES], (unsigned)cs.n_upd);
    atomicAdd(&s_ctr[CTR_HIST + min(cs.n_upd, 31)], 1u);
    atomicAdd(&s_ctr[CTR_EPS + cs.branch], 1u);
  }
  flush_stats<BLK>(s_ctr, d.ctr);
}

// Equilibrium initial condition of fluid cells in [c0, c0 + len): inputs are
// indexed by cell - c0; u planes are `us` elements apart.  Non-fluid cells in
// the range get zero populations and multipliers.
template <int BLK>
__global__ void __launch_bounds__(BLK) k_init(Desc d, const double* rho, const double* u,
                                              long long us, const double* T, long long c0,
                                              long long len, int maxit) {
  extern __shared__ double smem[];
  __shared__ unsigned int s_ctr[CTR_N];
  for (int k = threadIdx.x; k < CTR_N; k += BLK) s_ctr[k] = 0;
  __syncthreads();
  const long long r = (long long)blockIdx.x * BLK + threadIdx.x;
  const long long cell = c0 + r;
  if (r < len && cell < d.N) {
    const bool fluid = d.mask == nullptr || d.mask[cell] == MASK_FLUID;
    WS<BLK> w{smem + threadIdx.x};
    if (fluid) {
      const double rr = rho[r], ux = u[r], uy = u[us + r], uz = u[2 * us + r], TT = T[r];
      WS<BLK> lam = w.at(WS_LAM), F = w.at(WS_E), m = w.at(WS_M);
      targets<BLK>(ux, uy, uz, TT, m);
      gaussian_guess<BLK>(ux, uy, uz, TT, lam);
      const NewtonResult nr = newton<BLK>(lam, F, m, d.ph, maxit);
      const double cgr = d.ph.cg * TT * rr;
      static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        d.pop[(long long)i * d.Np + cell] = rr * F[i];
        d.pop[(long long)(Q + i) * d.Np + cell] = cgr * F[i];
      });
#pragma unroll
      for (int k = 0; k < NM; ++k) d.lam[k * d.Np + cell] = lam[k];
      atomicAdd(&s_ctr[CTR_FAILED], (unsigned)nr.failed);
    } else {
      for (int j = 0; j < 2 * Q; ++j) d.pop[(long long)j * d.Np + cell] = 0.0;
      for (int k = 0; k < NM; ++k) d.lam[k * d.Np + cell] = 0.0;
    }
  }
  flush_stats<BLK>(s_ctr, d.ctr);
}

// Equilibrium populations (f then g, 78 values) and multipliers of one state
// (rho, u, T), from a cold start; one thread.  Used for the far-field state.
template <int BLK>
__global__ void __launch_bounds__(BLK) k_state_equilibrium(Phys ph, double rho, double ux,
                                                           double uy, double uz, double T,
                                                           double* out78, int maxit,
                                                           unsigned long long* failed) {
  extern __shared__ double smem[];
  if (threadIdx.x != 0) return;
  WS<BLK> w{smem};
  WS<BLK> lam = w.at(WS_LAM), F = w.at(WS_E), m = w.at(WS_M);
  targets<BLK>(ux, uy, uz, T, m);
  gaussian_guess<BLK>(ux, uy, uz, T, lam);
  const NewtonResult nr = newton<BLK>(lam, F, m, ph, maxit);
  for (int i = 0; i < Q; ++i) {
    out78[i] = rho * F[i];
    out78[Q + i] = ph.cg * T * rho * F[i];
  }
  if (nr.failed) atomicAdd(failed, 1ull);
}

// After an even pass: freestream cells hold the far-field post-collision
// populations and outflow cells a copy of the cell with x clamped into
// [3, nx-4], both in the reversed (post-collision) layout the odd pass reads.
__global__ void k_fill_even(Desc d) {
  const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= d.N) return;
  const uint8_t mk = d.mask[cell];
  if (mk != MASK_FREE && mk != MASK_OUT) return;
  long long src = -1;
  if (mk == MASK_OUT) {
    const Coord c = coord_of(d, cell);
    const int xc = min(max(c.x, 3), d.nx - 4);
    src = cell + (xc - c.x);
    if (d.mask[src] == MASK_FREE) src = -1;
  }
  for (int i = 0; i < Q; ++i) {
    const long long jf = (long long)opp(i) * d.Np, jg = (long long)(Q + opp(i)) * d.Np;
    if (src < 0) {
      d.pop[jf + cell] = d.heq_inf[i];
      d.pop[jg + cell] = d.heq_inf[Q + i];
    } else {
      d.pop[jf + cell] = d.pop[jf + src];
      d.pop[jg + cell] = d.pop[jg + src];
    }
  }
}

// After an odd pass: fluid slots whose source is a freestream or outflow cell
// receive what that cell streamed: the far-field equilibrium, or the
// post-collision population of the clamped cell c (which c pushed into
// slot (c + xi_i, i), or bounced into (c, opp i) if c + xi_i is solid).
__global__ void k_fill_odd(Desc d) {
  const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= d.N || d.mask[cell] != MASK_FLUID) return;
  const Coord c = coord_of(d, cell);
  const bool near = (!d.per[0] && (c.x < 6 || c.x >= d.nx - 6)) ||
                    (!d.per[1] && (c.y < 6 || c.y >= d.ny - 6)) ||
                    (!d.per[2] && (c.z < 6 || c.z >= d.nz - 6));
  if (!near) return;
  const Nbr nb(d, c);
  for (int i = 0; i < Q; ++i) {
    const long long s = nb.at(-kCX[i], -kCY[i], -kCZ[i]);
    const uint8_t ms = d.mask[s];
    if (ms != MASK_FREE && ms != MASK_OUT) continue;
    const long long jf = (long long)i * d.Np, jg = (long long)(Q + i) * d.Np;
    long long src = -1;
    if (ms == MASK_OUT) {
      const Coord sc = coord_of(d, s);
      const int xc = min(max(sc.x, 3), d.nx - 4);
      const long long cc = s + (xc - sc.x);
      if (d.mask[cc] != MASK_FREE) {
        const Coord ccc = coord_of(d, cc);
        const long long t = (long long)wrap(ccc.x + kCX[i], d.nx) +
                            (long long)d.nx * (wrap(ccc.y + kCY[i], d.ny) +
                                               (long long)d.ny * wrap(ccc.z + kCZ[i], d.nz));
        src = (d.mask[t] == MASK_SOLID) ? (long long)opp(i) * d.Np + cc : jf + t;
      }
    }
    if (src < 0) {
      d.pop[jf + cell] = d.heq_inf[i];
      d.pop[jg + cell] = d.heq_inf[Q + i];
    } else {
      d.pop[jf + cell] = d.pop[src];
      d.pop[jg + cell] = d.pop[src + Q * d.Np];
    }
  }
}

// Moments of one cell's pre-collision populations: rho, u, T (total energy).
template <int BLK>
__device__ __forceinline__ void cell_macros(WS<BLK> w, double cv2inv, double& rho, double& ux,
                                            double& uy, double& uz, double& T) {
  double r = 0.0, jx = 0.0, jy = 0.0, jz = 0.0, e2 = 0.0;
  static_for<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const double fi = w[WS_F + i];
    r += fi;
    constexpr int cx = CX[i], cy = CY[i], cz = CZ[i], cc = c2(i);
    if constexpr (cx != 0) jx = fma((double)cx, fi, jx);
    if constexpr (cy != 0) jy = fma((double)cy, fi, jy);
    if constexpr (cz != 0) jz = fma((double)cz, fi, jz);
    if constexpr (cc != 0) e2 = fma((double)cc, fi, e2);
    e2 += w[WS_G + i];
  });
  const double ir = 1.0 / r;
  rho = r;
  ux = jx * ir; uy = jy * ir; uz = jz * ir;
  T = (e2 - r * (ux * ux + uy * uy + uz * uz)) * cv2inv * ir;
}

// rho, u, T, p = rho T of cells [c0, c0 + len) into out arrays indexed by
// cell - c0 (u planes `us` apart; any pointer may be null); non-fluid cells 0.
template <bool ODD, int BLK>
__global__ void __launch_bounds__(BLK) k_macros(Desc d, double* rho, double* u, long long us,
                                                double* T, double* p, long long c0,
                                                long long len) {
  extern __shared__ double smem[];
  const long long r = (long long)blockIdx.x * BLK + threadIdx.x;
  const long long cell = c0 + r;
  if (r >= len || cell >= d.N) return;
  double vr = 0, vx = 0, vy = 0, vz = 0, vT = 0;
  if (d.mask == nullptr || d.mask[cell] == MASK_FLUID) {
    WS<BLK> w{smem + threadIdx.x};
    gather<ODD, BLK>(d, cell, w);
    cell_macros<BLK>(w, d.ph.inv_2cv, vr, vx, vy, vz, vT);
  }
  if (rho) rho[r] = vr;
  if (u) { u[r] = vx; u[us + r] = vy; u[2 * us + r] = vz; }
  if (T) T[r] = vT;
  if (p) p[r] = vr * vT;
}

// Conserved sums over fluid cells (mass, momentum, total energy): fixed
// grid-stride assignment and fixed-order tree reductions, so the result is
// deterministic.  partials: gridDim.x * 5 doubles.
template <bool ODD, int BLK>
__global__ void __launch_bounds__(BLK) k_conserved(Desc d, double* partials) {
  extern __shared__ double smem[];
  __shared__ double red[5][BLK];
  double acc[5] = {0, 0, 0, 0, 0};
  WS<BLK> w{smem + threadIdx.x};
  for (long long cell = (long long)blockIdx.x * BLK + threadIdx.x; cell < d.N;
       cell += (long long)gridDim.x * BLK) {
    if (d.mask != nullptr && d.mask[cell] != MASK_FLUID) continue;
    gather<ODD, BLK>(d, cell, w);
    static_for<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      const double fi = w[WS_F + i];
      constexpr int cx = CX[i], cy = CY[i], cz = CZ[i], cc = c2(i);
      acc[0] += fi;
      acc[1] += cx * fi;
      acc[2] += cy * fi;
      acc[3] += cz * fi;
      acc[4] += 0.5 * (cc * fi + w[WS_G + i]);
    });
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int s = BLK / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
#pragma unroll
      for (int k = 0; k < 5; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 5) partials[blockIdx.x * 5 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void k_sum_partials(const double* partials, int nblocks, double* out5) {
  const int k = threadIdx.x;
  if (k >= 5) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += partials[b * 5 + k];
  out5[k] = s;
}

}  // namespace lbm39
