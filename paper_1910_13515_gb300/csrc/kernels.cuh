// kernels.cuh -- CUDA kernels of the D3Q39 DDF step: initial equilibrium, the
// fused collide-and-stream passes (AA pattern), boundary fills, macroscopic
// read-out and conserved sums.
//
// Storage: 78 planes of Np elements (f_0..f_38 then g_0..g_38), x fastest,
// of type P: double (FP64 path) or float (precision form: each population
// stored as its deviation from a reference population h_ref, Desc::href).
// AA pattern over one buffer.  At even time the buffer holds the
// pre-collision populations h_i(x) in slot (x, i).  The even pass reads its
// own slots, collides and writes h*_i(x) into slot (x, opp i).  The odd pass
// gathers h_i(x) = h*_i(x - xi_i) from slot (x - xi_i, opp i), collides and
// pushes h*_i(x) into slot (x + xi_i, i), which is the pre-collision h_i of
// the next time step.  Every slot is read and written by one thread only (the
// slot pushed for direction i is the one gathered for opp(i)).  Solid,
// freestream and outflow cells never collide.  After each pass the fill
// kernels write into the slots of those cells (and, after an odd pass, of
// their fluid neighbours) what the fluid cells read next: the half-way
// bounce-back copies of solid cells and what freestream and outflow cells
// would have streamed (Sec. 4 boundary kinds), so the step kernels treat
// every neighbour alike.
//
// A fluid cell's step runs in three phases: gather and moments; targets and
// Newton (F, lam, m in shared memory); gather again, sensor, BGK and push.
#pragma once
#include <cstdint>

#include "cell.cuh"

namespace lbm39 {

struct Desc {
  void* pop;                          // 78 planes of P
  double* lam;                        // 13 planes of multipliers kept between steps, then
                                      // 39 planes of F_i = exp(Phi lam) at them
  const uint8_t* mask;                // nullptr: every cell fluid, all axes periodic
  unsigned long long* ctr;            // counters (CTR_*)
  const void* free_store;             // 78 stored values (P) of a freestream cell
  const double* heq_inf;              // 78 far-field equilibrium populations (FP64)
  const double* href;                 // 78 reference populations (precision form)
  double mref[5];                     // sum of href: rho, j, sum f|xi|^2 + sum g
  long long N, Np;                    // cells, plane stride in elements
  long long t;                        // time step being taken (schedules fallback retries)
  int d2;                             // one cell thick in z, z-mirror-symmetric populations
  int nx, ny, nz;
  int per[3];                         // periodic axes
  Phys ph;
};

// CTR_UPD32: float steps of single-precision starts; CTR_START32: solves that took one.
enum {
  CTR_FAILED = 0, CTR_UPDATES = 1, CTR_HIST = 2, CTR_EPS = 34, CTR_UPD32 = 38, CTR_START32 = 39,
  CTR_N = 40
};
// Set by lbm39_init when some fluid cell starts with u_z != 0 (outside the
// block counters: not reported by lbm39_stats).
constexpr int CTR_ASYM = 42;

struct Coord {
  int x, y, z;
};

// (cell < 2^31: lattices are limited to 2^31 - 1 cells)
__device__ __forceinline__ Coord coord_of(const Desc& d, long long cell) {
  const int c = (int)cell;
  const int yz = c / d.nx;
  return Coord{c - yz * d.nx, yz % d.ny, yz / d.ny};
}

// a mod n for a in [-3, n + 2]: one conditional correction when n >= 3.
__device__ __forceinline__ int wrap(int a, int n) {
  if (n >= 3) return a < 0 ? a + n : (a >= n ? a - n : a);
  const int r = a % n;
  return r < 0 ? r + n : r;
}

// Index of the cell at x + (dx, dy, dz) with periodic wrap of every axis
// (non-periodic axes carry boundary layers, so fluid cells never wrap there).
// Every index is below 2^31, so the 21 terms are 32-bit.
struct Nbr {
  int xs[7], ys[7], zs[7];
  __device__ __forceinline__ Nbr() {}
  __device__ __forceinline__ Nbr(const Desc& d, Coord c) {
#pragma unroll
    for (int s = 0; s < 7; ++s) {
      xs[s] = wrap(c.x + s - 3, d.nx);
      ys[s] = wrap(c.y + s - 3, d.ny) * d.nx;
      zs[s] = wrap(c.z + s - 3, d.nz) * d.nx * d.ny;
    }
  }
  __device__ __forceinline__ int at(int dx, int dy, int dz) const {
    return xs[dx + 3] + ys[dy + 3] + zs[dz + 3];
  }
};

// The neighbour table of the cell at c, built from a copy of the coordinates
// that the compiler cannot see through: a table built before the constraint
// solve is then not kept in registers across it (the odd pass builds it twice).
template <bool ODD>
__device__ __forceinline__ Nbr fresh_nbr(const Desc& d, Coord c) {
  Nbr nb;
  if constexpr (ODD) {
    asm volatile("" : "+r"(c.x), "+r"(c.y), "+r"(c.z));
    nb = Nbr(d, c);
  }
  return nb;
}

// Pre-collision populations of one distribution (base 0: f, Q: g) of fluid
// cell `cell` at the lattice's current time: own slots at even time, the odd
// gather from (x - xi_i, slot opp i) at odd time.  Where x - xi_i is solid,
// that slot holds the bounced population (bounce_even_cell), so the gather
// has no per-direction branch.
template <bool ODD, class P>
__device__ __forceinline__ void gather(const Desc& d, long long cell, const Nbr& nb, int base,
                                       P (&h)[Q]) {
  const P* __restrict__ pop = static_cast<const P*>(d.pop);
  static_for<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if constexpr (!ODD) {
      h[i] = pop[(long long)(base + i) * d.Np + cell];
    } else {
      constexpr int cx = CX[i], cy = CY[i], cz = CZ[i];
      h[i] = pop[(long long)(base + opp(i)) * d.Np + nb.at(-cx, -cy, -cz)];
    }
  });
}

// Post-collision population h*_i of fluid cell `cell` into its AA slot: own
// slot opp i at even time, (x + xi_i, slot i) at odd time (a solid x + xi_i
// hands it back to x afterwards: bounce_odd_cell).
template <bool ODD, class P, int i>
__device__ __forceinline__ void push(const Desc& d, long long cell, const Nbr& nb, int base,
                                     P v) {
  P* __restrict__ pop = static_cast<P*>(d.pop);
  if constexpr (!ODD) {
    pop[(long long)(base + opp(i)) * d.Np + cell] = v;
  } else {
    constexpr int cx = CX[i], cy = CY[i], cz = CZ[i];
    pop[(long long)(base + i) * d.Np + nb.at(cx, cy, cz)] = v;
  }
}

// Raw moments of a cell: rho, j = rho u, e2 = sum f|xi|^2 + sum g = 2 rho E.
struct Raw {
  double rho, jx, jy, jz, e2;
};

// Phase A: gather each distribution in turn and take the moments (FP64).
template <bool ODD, class P>
__device__ __forceinline__ Raw gather_raw(const Desc& d, long long cell, const Nbr& nb) {
  Raw r;
  double gs;
  if constexpr (sizeof(P) == 8) {
    P h[Q];
    gather<ODD, P>(d, cell, nb, 0, h);
    gen::f_moments<double>(h, r.rho, r.jx, r.jy, r.jz, r.e2);
    gather<ODD, P>(d, cell, nb, Q, h);
    gs = gen::g_sum<double>(h);
  } else {  // deviations: moments of h_ref (precomputed) plus those of the deviations
    P h[Q];
    double hd[Q];
    gather<ODD, P>(d, cell, nb, 0, h);
#pragma unroll
    for (int i = 0; i < Q; ++i) hd[i] = (double)h[i];
    gen::f_moments<double>(hd, r.rho, r.jx, r.jy, r.jz, r.e2);
    gather<ODD, P>(d, cell, nb, Q, h);
#pragma unroll
    for (int i = 0; i < Q; ++i) hd[i] = (double)h[i];
    gs = gen::g_sum<double>(hd);
    r.rho += d.mref[0]; r.jx += d.mref[1]; r.jy += d.mref[2]; r.jz += d.mref[3];
    gs += d.mref[4];
  }
  r.e2 += gs;
  return r;
}

template <bool ODD, class P>
__device__ __forceinline__ Macro gather_moments(const Desc& d, long long cell, const Nbr& nb) {
  const Raw r = gather_raw<ODD, P>(d, cell, nb);
  return macro_from_moments(r.rho, r.jx, r.jy, r.jz, r.e2, d.ph.inv_2cv);
}

// Phase C: gather again, Knudsen sensor (Eq. DeltaAvg, f only), tau_eff =
// tau alpha(eps) (Eq. alpha) for f and g, BGK and push.  F holds the final
// normalised equilibrium; f^eq = rho F, g^eq = (2C_v - D) T rho F.
// PR: with the Prandtl-number adjustment (the quasi-equilibrium correction of g;
// a separate instantiation, so the paper's Pr = 1 collision carries none of it).
template <bool ODD, class P, int BLK, bool PR = false>
__device__ __forceinline__ int relax_push(const Desc& d, long long cell, const Nbr& nb,
                                          const Macro& M, WS<BLK> F) {
  const Phys& ph = d.ph;
  const double rho = M.rho;
  const float rho32 = trunc_float(rho);
  const double cgr = ph.cg * M.T * rho;
  double eps;
  if constexpr (sizeof(P) == 8) {
    P f[Q];
    gather<ODD, P>(d, cell, nb, 0, f);
    // FP32 screen of 39 eps from float views (error bound: screen_undecided);
    // the FP64 value where the screen cannot decide the branch of Eq. (alpha)
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    int emin = SCREEN_EMAX, emax = SCREEN_EMIN;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const double Fd = F[i];
      const int eF = exp_field(Fd), ef = exp_field(f[i]);
      emin = min(emin, min(eF, ef));
      emax = max(emax, max(eF, ef));
      const float feq = rho32 * view_float(Fd);
      acc[i & 3] += fabsf(view_float(f[i]) - feq) * rcp32(feq);
    }
    const float s32 = (acc[0] + acc[1]) + (acc[2] + acc[3]);
    eps = (double)s32 * (1.0 / Q);
    if (screen_undecided(s32, emin, emax, rho32)) {
      double s = 0.0;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const double feq = rho * F[i];
        s += fabs(f[i] - feq) / feq;
      }
      eps = s * (1.0 / Q);
    }
    const int branch = alpha_branch(eps);
    const double omega = omega_of(ph, branch);
    static_for<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      push<ODD, P, i>(d, cell, nb, 0, fma(-omega, fma(-rho, F[i], f[i]), f[i]));
    });
    double s13[NM];
    if constexpr (PR) gen::moments_s<double>(f, s13);  // sum_i f_i phi_k(xi_i)
    P g[Q];
    gather<ODD, P>(d, cell, nb, Q, g);
    if constexpr (!PR) {
      static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        push<ODD, P, i>(d, cell, nb, Q, fma(-omega, fma(-cgr, F[i], g[i]), g[i]));
      });
    } else {
      // heat flux q = (1/2) sum_i c_i (|c_i|^2 f_i + g_i), c_i = xi_i - u, from the raw
      // sums: sum_i f_i c_i |c_i|^2 = S3 - 2 S2 u - u sum_i f_i |xi_i|^2 + 2 rho u |u|^2
      const double ux = M.ux, uy = M.uy, uz = M.uz, u2 = ux * ux + uy * uy + uz * uz;
      const double e2f = s13[4] + s13[5] + s13[6];
      double g0 = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
      static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int cx = CX[i], cy = CY[i], cz = CZ[i];
        g0 += g[i];
        if constexpr (cx != 0) gx = fma((double)cx, g[i], gx);
        if constexpr (cy != 0) gy = fma((double)cy, g[i], gy);
        if constexpr (cz != 0) gz = fma((double)cz, g[i], gz);
      });
      const double r2u2 = 2.0 * s13[0] * u2;
      const double qx = 0.5 * (s13[10] - 2.0 * (s13[4] * ux + s13[7] * uy + s13[8] * uz) -
                               ux * e2f + r2u2 * ux + gx - ux * g0);
      const double qy = 0.5 * (s13[11] - 2.0 * (s13[7] * ux + s13[5] * uy + s13[9] * uz) -
                               uy * e2f + r2u2 * uy + gy - uy * g0);
      const double qz = 0.5 * (s13[12] - 2.0 * (s13[8] * ux + s13[9] * uy + s13[6] * uz) -
                               uz * e2f + r2u2 * uz + gz - uz * g0);
      // (1/tau - 1/tau2) g^eq_i (c_i . b), b = 2 q / ((2 C_v - D) rho T^2),
      // = F_i (beta0 + xi_i . beta) with beta = 2 (1/tau - 1/tau2) q / T, beta0 = -u . beta
      const double k = 2.0 * domega_of(ph, branch) / M.T;
      const double bx = k * qx, by = k * qy, bz = k * qz;
      const double b0 = -(ux * bx + uy * by + uz * bz);
      static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int cx = CX[i], cy = CY[i], cz = CZ[i];
        const double cb = fma((double)cx, bx, fma((double)cy, by, fma((double)cz, bz, b0)));
        push<ODD, P, i>(d, cell, nb, Q,
                        fma(F[i], cb, fma(-omega, fma(-cgr, F[i], g[i]), g[i])));
      });
    }
  } else {
    // precision form: h~ = h - h_ref stored in FP32; equilibrium deviation
    // h^eq - h_ref formed in FP64 and rounded; sensor and BGK in FP32.
    // The sensor compares each stored deviation with the equilibrium in the same storage,
    // rf_i = (f^eq_i - f_ref_i) rounded to float: s = 39 eps = sum_i |f~_i - rf_i| / f^eq_i.
    // FP32 screen, and the FP64 value of the same sum where the screen cannot decide the
    // branch of Eq. (alpha) (screen_undecided_dev), so alpha is an FP64 decision.
    const double* __restrict__ href = d.href;
    P f[Q];
    gather<ODD, P>(d, cell, nb, 0, f);
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const double Fi = F[i];
      f[i] -= __double2float_rn(fma(rho, Fi, -__ldg(href + i)));  // f~ - (f^eq - f_ref)
      acc[i & 3] += fabsf(f[i]) * rcp32(rho32 * trunc_float(Fi));
    }
    const float s32 = (acc[0] + acc[1]) + (acc[2] + acc[3]);
    eps = (double)s32 * (1.0 / Q);
    if (screen_undecided_dev(s32)) {
      P fs[Q];
      gather<ODD, P>(d, cell, nb, 0, fs);  // the stored values (cached)
      double s = 0.0;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const double feq = rho * F[i];
        const float rf = __double2float_rn(fma(rho, F[i], -__ldg(href + i)));
        s += fabs((double)fs[i] - (double)rf) / feq;  // the difference is exact
      }
      eps = s * (1.0 / Q);
    }
    const float omega = (float)omega_of(ph, alpha_branch(eps));
    P f2[Q];
    gather<ODD, P>(d, cell, nb, 0, f2);  // the stored values again (cached)
    static_for<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      push<ODD, P, i>(d, cell, nb, 0, fmaf(-omega, f[i], f2[i]));
    });
    P g[Q];
    gather<ODD, P>(d, cell, nb, Q, g);
    if constexpr (!PR) {
      static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const float qg = __double2float_rn(fma(cgr, F[i], -__ldg(href + Q + i)));
        push<ODD, P, i>(d, cell, nb, Q, fmaf(-omega, g[i] - qg, g[i]));
      });
    } else {
      // heat flux from the non-equilibrium parts (the 13-moment equilibrium has none):
      // q = (1/2) sum_i c_i (|c_i|^2 (f_i - f^eq_i) + (g_i - g^eq_i)), in FP32
      const float ux = (float)M.ux, uy = (float)M.uy, uz = (float)M.uz;
      float e[Q], qx = 0.0f, qy = 0.0f, qz = 0.0f;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        e[i] = g[i] - __double2float_rn(fma(cgr, F[i], -__ldg(href + Q + i)));  // g - g^eq
        const float cx = (float)kCX[i] - ux, cy = (float)kCY[i] - uy, cz = (float)kCZ[i] - uz;
        const float w = 0.5f * fmaf(cx * cx + cy * cy + cz * cz, f[i], e[i]);
        qx = fmaf(cx, w, qx);
        qy = fmaf(cy, w, qy);
        qz = fmaf(cz, w, qz);
      }
      const float k = (float)(2.0 * domega_of(ph, alpha_branch(eps)) / M.T);
      const float bx = k * qx, by = k * qy, bz = k * qz;
      const float b0 = -(ux * bx + uy * by + uz * bz);
      static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int cx = CX[i], cy = CY[i], cz = CZ[i];
        const float cb = fmaf((float)cx, bx, fmaf((float)cy, by, fmaf((float)cz, bz, b0)));
        push<ODD, P, i>(d, cell, nb, Q, fmaf(trunc_float(F[i]), cb, fmaf(-omega, e[i], g[i])));
      });
    }
  }
  return alpha_branch(eps);
}

template <int BLK>
__device__ __forceinline__ void flush_stats(unsigned int* s_ctr, unsigned long long* ctr) {
  __syncthreads();
  for (int k = threadIdx.x; k < CTR_N; k += BLK)
    if (s_ctr[k]) atomicAdd(ctr + k, (unsigned long long)s_ctr[k]);
}

// Per-cell solver state between steps: lam (13 planes) and F = exp(Phi lam)
// (39 planes), in that order from Desc::lam.
constexpr int SOLVER_PLANES = NM + Q;

template <int BLK>
__device__ __forceinline__ void load_solver_state(const Desc& d, long long cell, WS<BLK> w) {
  const double* __restrict__ st = d.lam;
#pragma unroll
  for (int k = 0; k < NM; ++k) w[WS_LAM + k] = st[k * d.Np + cell];
#pragma unroll
  for (int i = 0; i < Q; ++i) w[WS_E + i] = st[(NM + i) * d.Np + cell];
}

template <int BLK>
__device__ __forceinline__ void store_solver_state(const Desc& d, long long cell, WS<BLK> w) {
  double* __restrict__ st = d.lam;
#pragma unroll
  for (int k = 0; k < NM; ++k) st[k * d.Np + cell] = w[WS_LAM + k];
#pragma unroll
  for (int i = 0; i < Q; ++i) st[(NM + i) * d.Np + cell] = w[WS_E + i];
}

// F = exp(Phi lam) at the workspace multipliers.
template <int BLK>
__device__ __forceinline__ void eval_at_lam(WS<BLK> w) {
  double G[NM];
  eval_equilibrium<BLK>(w.at(WS_LAM), w.at(WS_DL), 0.0, w.at(WS_E), w.at(WS_M), G, false);
}

// Where the 13-moment solve failed or took no update: the fallback's
// multipliers embedded in lam and marked (lam unchanged but unmarked if the
// fallback fails too), and F = exp(Phi lam) exactly as the full solve
// evaluates it (the fallback evaluates the embedding with the same exponents
// and exponential), so the cached F stays exact.  retry:
// the cell came in with a fallback embedding, whose five multipliers (still in
// the stored state) start the fallback.
// state, Np: the solver-state planes (Desc::lam) and their stride.
template <int BLK>
__device__ __noinline__ void fallback_cell(const double* state, long long Np, long long cell,
                                           WS<BLK> w, double T, bool retry) {
  double warm[N5];
  if (retry) {
#pragma unroll
    for (int k = 0; k < N5; ++k) warm[k] = state[k * Np + cell];
  }
  WS<BLK> lam = w.at(WS_LAM);
  if (fallback_equilibrium<BLK>(w, T, retry ? warm : nullptr) == 0) {
    WS<BLK> mu = w.at(WS_M);
#pragma unroll
    for (int k = 0; k < 4; ++k) lam[k] = mu[k];
    lam[4] = lam[5] = lam[6] = mu[4];
#pragma unroll
    for (int k = 7; k < NM; ++k) lam[k] = 0.0;
    lam[9] = -0.0;  // the embedding mark: on the fallback
    // F already holds exp(Phi lam): the fallback's last evaluation was at this
    // embedding, with the full solve's exponents and exponential
  } else {
    lam[9] = lam[9] + 0.0;  // the fallback failed too: not on the fallback
    eval_at_lam<BLK>(w);    // F = exp(Phi lam), the cached value the next solve starts from
  }
}

// Newton budget of a cell on the fallback at time step t: the full budget
// maxit on the steps that are multiples of RETRY_PERIOD, else none.
__device__ __forceinline__ int retry_budget(long long t, int maxit) {
  return (t & (RETRY_PERIOD - 1)) == 0 ? maxit : 0;
}

// The constraint solve of a cell from the warm start in the workspace (F cached
// at lam) with the lattice's root finder SOLVER (FP64 path): 0 Newton-Raphson;
// 1 the chord-Newton hybrid (newton_chord); 2 Newton with a single-precision
// direction (newton<BLK, true>); 3 that after a single-precision start
// (start32).  The precision form (P = float) always takes 3.  n32: the float
// steps of the start.
template <class P, int BLK, bool D2, int SOLVER>
__device__ __forceinline__ NewtonResult solve_cell(WS<BLK> w, const Phys& ph, int maxit,
                                                   int& n32) {
  n32 = 0;
  if constexpr (SOLVER == 1 && sizeof(P) == 8) {
    return newton_chord<BLK, D2>(w, ph, maxit, true);
  } else {
    bool cached = true;
    if constexpr (sizeof(P) == 4 || SOLVER == 3) {
      if (maxit > 0) {  // a cell on the fallback off a retry step takes no step at all
        n32 = start32<BLK, D2>(w);
        cached = n32 == 0;
      }
    }
    return newton<BLK, sizeof(P) == 4 || SOLVER >= 2, D2>(w, ph, maxit, cached);
  }
}

// One fluid cell's time step (even or odd AA pass): phases A, B and C, with
// the Newton statistics added to the block's counters.  w: the cell's workspace.
// D2: the nine-function constraint system of a z-mirror-symmetric lattice one
// cell thick in z (Sys<true>; the same values as the full system).
// SOLVER: the root finder of the constraint equations (solve_cell).
template <bool ODD, class P, int BLK, bool D2 = false, bool PR = false, int SOLVER = 0>
__device__ __forceinline__ void step_cell(const Desc& d, long long cell, WS<BLK> w,
                                          unsigned int* s_ctr) {
  WS<BLK> F = w.at(WS_E), lam = w.at(WS_LAM), m = w.at(WS_M);
  Coord c{0, 0, 0};
  if constexpr (ODD) c = coord_of(d, cell);
  const Macro M = gather_moments<ODD, P>(d, cell, fresh_nbr<ODD>(d, c));
  targets<BLK>(M.ux, M.uy, M.uz, M.T, m);
  load_solver_state<BLK>(d, cell, w);
  const bool marked = is_fallback_embedding<BLK>(lam);
  // a marked cell off a retry step gets no update (it stays on the fallback
  // unless its embedding already meets the 13 constraints)
  const int maxit = !marked ? d.ph.maxit : retry_budget(d.t, d.ph.maxit);
  int n32;
  const NewtonResult nr = solve_cell<P, BLK, D2, SOLVER>(w, d.ph, maxit, n32);
  if (nr.failed) fallback_cell<BLK>(d.lam, d.Np, cell, w, M.T, marked);
  else lam[9] = lam[9] + 0.0;  // a solved state carries no embedding mark
  store_solver_state<BLK>(d, cell, w);
  const int branch = relax_push<ODD, P, BLK, PR>(d, cell, fresh_nbr<ODD>(d, c), M, F);
  atomicAdd(&s_ctr[CTR_FAILED], (unsigned)nr.failed);
  atomicAdd(&s_ctr[CTR_UPDATES], (unsigned)nr.n_upd);
  atomicAdd(&s_ctr[CTR_HIST + min(nr.n_upd, 31)], 1u);
  atomicAdd(&s_ctr[CTR_EPS + branch], 1u);
  if (n32) {
    atomicAdd(&s_ctr[CTR_UPD32], (unsigned)n32);
    atomicAdd(&s_ctr[CTR_START32], 1u);
  }
}

// One time step over every fluid cell (even or odd AA pass).
template <bool ODD, class P, int BLK, bool D2, bool PR = false, int SOLVER = 0>
__global__ void __launch_bounds__(BLK) k_step(Desc d) {
  extern __shared__ double smem[];
  __shared__ unsigned int s_ctr[CTR_N];
  for (int k = threadIdx.x; k < CTR_N; k += BLK) s_ctr[k] = 0;
  load_exp_table();
  const long long cell = (long long)blockIdx.x * BLK + threadIdx.x;
  if (cell < d.N && (d.mask == nullptr || d.mask[cell] == MASK_FLUID))
    step_cell<ODD, P, BLK, D2, PR, SOLVER>(d, cell, WS<BLK>{smem + threadIdx.x}, s_ctr);
  flush_stats<BLK>(s_ctr, d.ctr);
}

// Stored value of population j (0..77) whose FP64 value is v.
template <class P>
__device__ __forceinline__ P to_store(const Desc& d, int j, double v) {
  if constexpr (sizeof(P) == 8) return v;
  else return __double2float_rn(v - __ldg(d.href + j));
}

// Equilibrium initial condition of fluid cells in [c0, c0 + len): inputs are
// indexed by cell - c0; u planes are `us` elements apart.  Non-fluid cells in
// the range get zero populations and multipliers.
template <class P, int BLK>
__global__ void __launch_bounds__(BLK) k_init(Desc d, const double* rho, const double* u,
                                              long long us, const double* T, long long c0,
                                              long long len, int maxit) {
  extern __shared__ double smem[];
  __shared__ unsigned int s_ctr[CTR_N];
  for (int k = threadIdx.x; k < CTR_N; k += BLK) s_ctr[k] = 0;
  load_exp_table();
  const long long r = (long long)blockIdx.x * BLK + threadIdx.x;
  const long long cell = c0 + r;
  P* pop = static_cast<P*>(d.pop);
  int asym = 0;
  if (r < len && cell < d.N) {
    const bool fluid = d.mask == nullptr || d.mask[cell] == MASK_FLUID;
    WS<BLK> w{smem + threadIdx.x};
    if (fluid) {
      const double rr = rho[r], ux = u[r], uy = u[us + r], uz = u[2 * us + r], TT = T[r];
      asym = uz != 0.0;
      WS<BLK> lam = w.at(WS_LAM), F = w.at(WS_E), m = w.at(WS_M);
      targets<BLK>(ux, uy, uz, TT, m);
      gaussian_guess<BLK>(ux, uy, uz, TT, lam);
      const NewtonResult nr = newton<BLK, false>(w, d.ph, maxit, false);
      if (nr.failed) fallback_cell<BLK>(d.lam, d.Np, cell, w, TT, false);
      store_solver_state<BLK>(d, cell, w);
      const double cgr = d.ph.cg * TT * rr;
      for (int i = 0; i < Q; ++i) {
        pop[(long long)i * d.Np + cell] = to_store<P>(d, i, rr * F[i]);
        pop[(long long)(Q + i) * d.Np + cell] = to_store<P>(d, Q + i, cgr * F[i]);
      }
      atomicAdd(&s_ctr[CTR_FAILED], (unsigned)nr.failed);
    } else {
      for (int j = 0; j < 2 * Q; ++j) pop[(long long)j * d.Np + cell] = P(0);
      for (int k = 0; k < SOLVER_PLANES; ++k) d.lam[k * d.Np + cell] = 0.0;
    }
  }
  if (__syncthreads_or(asym) && threadIdx.x == 0) atomicAdd(d.ctr + CTR_ASYM, 1ull);
  flush_stats<BLK>(s_ctr, d.ctr);
}

// Equilibrium populations (f then g, 78 values) and multipliers of one state
// (rho, u, T), from a cold start; one thread.  Used for the far-field state
// and for the reference state of the precision form.
template <int BLK>
__global__ void __launch_bounds__(BLK) k_state_equilibrium(Phys ph, double rho, double ux,
                                                           double uy, double uz, double T,
                                                           double* out78, int maxit,
                                                           unsigned long long* failed) {
  extern __shared__ double smem[];
  load_exp_table();
  if (threadIdx.x != 0) return;
  WS<BLK> w{smem};
  WS<BLK> lam = w.at(WS_LAM), F = w.at(WS_E), m = w.at(WS_M);
  targets<BLK>(ux, uy, uz, T, m);
  gaussian_guess<BLK>(ux, uy, uz, T, lam);
  const NewtonResult nr = newton<BLK, false>(w, ph, maxit, false);
  for (int i = 0; i < Q; ++i) {
    out78[i] = rho * F[i];
    out78[Q + i] = ph.cg * T * rho * F[i];
  }
  if (nr.failed) atomicAdd(failed, 1ull);
}

// A population reversed by the bounce-back: the stored value v of population
// `from` becomes population `to`.  FP64 storage holds the populations
// themselves; the precision form holds deviations from the reference
// populations, which differ between the two directions unless the reference
// is at rest, so the value is re-referenced: (v + h_ref,from) - h_ref,to.
template <class P>
__device__ __forceinline__ P reversed(const Desc& d, P v, int from, int to) {
  if constexpr (sizeof(P) == 8) return v;
  else return __double2float_rn((double)v + (__ldg(d.href + from) - __ldg(d.href + to)));
}

// After an even pass: freestream cells hold the far-field post-collision
// populations and outflow cells a copy of the cell with x clamped into
// [3, nx-4], both in the reversed (post-collision) layout the odd pass reads.
// Half-way bounce-back (Sec. 4) after an even pass.  The even pass leaves
// f*_opp(i)(x) of a fluid cell x in its slot i; the odd pass gathers f_i(x)
// from (x - xi_i, slot opp i), which for x = s + xi_i is (s, slot opp i): the
// solid cell s copies the value there.  Each of these slots has one writer.
template <class P>
__device__ __forceinline__ void bounce_even_cell(const Desc& d, long long s) {
  P* pop = static_cast<P*>(d.pop);
  const Nbr nb(d, coord_of(d, s));
  for (int i = 0; i < Q; ++i) {
    const long long x = nb.at(kCX[i], kCY[i], kCZ[i]);
    if (d.mask[x] != MASK_FLUID) continue;
    const int o = opp(i);  // slot i of x holds population o of x; it returns as population i
    pop[(long long)o * d.Np + s] = reversed<P>(d, pop[(long long)i * d.Np + x], o, i);
    pop[(long long)(Q + o) * d.Np + s] =
        reversed<P>(d, pop[(long long)(Q + i) * d.Np + x], Q + o, Q + i);
  }
}

// Half-way bounce-back after an odd pass: fluid cell x = s - xi_i pushed
// f*_i(x) into (s, slot i); it returns as f_opp(i)(x), which the even pass
// reads from (x, slot opp i) -- a slot no push writes, since its source
// x - xi_opp(i) = s is solid.
template <class P>
__device__ __forceinline__ void bounce_odd_cell(const Desc& d, long long s) {
  P* pop = static_cast<P*>(d.pop);
  const Nbr nb(d, coord_of(d, s));
  for (int i = 0; i < Q; ++i) {
    const long long x = nb.at(-kCX[i], -kCY[i], -kCZ[i]);
    if (d.mask[x] != MASK_FLUID) continue;
    const int o = opp(i);  // population i of x returns as its population o
    pop[(long long)o * d.Np + x] = reversed<P>(d, pop[(long long)i * d.Np + s], i, o);
    pop[(long long)(Q + o) * d.Np + x] =
        reversed<P>(d, pop[(long long)(Q + i) * d.Np + s], Q + i, Q + o);
  }
}

template <class P>
__device__ __forceinline__ void fill_even_cell(const Desc& d, long long cell) {
  const uint8_t mk = d.mask[cell];
  if (mk == MASK_SOLID) {
    bounce_even_cell<P>(d, cell);
    return;
  }
  if (mk != MASK_FREE && mk != MASK_OUT) return;
  P* pop = static_cast<P*>(d.pop);
  const P* fs = static_cast<const P*>(d.free_store);
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
      pop[jf + cell] = fs[i];
      pop[jg + cell] = fs[Q + i];
    } else {
      pop[jf + cell] = pop[jf + src];
      pop[jg + cell] = pop[jg + src];
    }
  }
}

// After an odd pass: fluid slots whose source is a freestream or outflow cell
// receive what that cell streamed: the far-field equilibrium, or the
// post-collision population of the clamped cell c, which c pushed into slot
// (c + xi_i, i) (also when c + xi_i is solid: bounce_odd_cell only copies it
// on).  Solid cells do their bounce-back copies.
template <class P>
__device__ __forceinline__ void fill_odd_cell(const Desc& d, long long cell) {
  const uint8_t mk = d.mask[cell];
  if (mk == MASK_SOLID) {
    bounce_odd_cell<P>(d, cell);
    return;
  }
  if (mk != MASK_FLUID) return;
  const Coord c = coord_of(d, cell);
  const bool near = (!d.per[0] && (c.x < 6 || c.x >= d.nx - 6)) ||
                    (!d.per[1] && (c.y < 6 || c.y >= d.ny - 6)) ||
                    (!d.per[2] && (c.z < 6 || c.z >= d.nz - 6));
  if (!near) return;
  P* pop = static_cast<P*>(d.pop);
  const P* fs = static_cast<const P*>(d.free_store);
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
        src = jf + t;
      }
    }
    if (src < 0) {
      pop[jf + cell] = fs[i];
      pop[jg + cell] = fs[Q + i];
    } else {
      pop[jf + cell] = pop[src];
      pop[jg + cell] = pop[src + Q * d.Np];
    }
  }
}

template <class P>
__global__ void k_fill_even(Desc d) {
  const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell < d.N) fill_even_cell<P>(d, cell);
}

template <class P>
__global__ void k_fill_odd(Desc d) {
  const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell < d.N) fill_odd_cell<P>(d, cell);
}

// rho, u, T, p = rho T of cells [c0, c0 + len) into out arrays indexed by
// cell - c0 (u planes `us` apart; any pointer may be null); non-fluid cells 0.
template <bool ODD, class P>
__global__ void k_macros(Desc d, double* rho, double* u, long long us, double* T, double* p,
                         long long c0, long long len) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long cell = c0 + r;
  if (r >= len || cell >= d.N) return;
  Macro M{0, 0, 0, 0, 0};
  if (d.mask == nullptr || d.mask[cell] == MASK_FLUID) {
    Nbr nb;
    if constexpr (ODD) nb = Nbr(d, coord_of(d, cell));
    M = gather_moments<ODD, P>(d, cell, nb);
  }
  if (rho) rho[r] = M.rho;
  if (u) { u[r] = M.ux; u[us + r] = M.uy; u[2 * us + r] = M.uz; }
  if (T) T[r] = M.T;
  if (p) p[r] = M.rho * M.T;
}

// Conserved sums over fluid cells (mass, momentum, total energy): fixed
// grid-stride assignment and fixed-order tree reductions, so the result is
// deterministic.  partials: gridDim.x * 5 doubles.
template <bool ODD, class P, int BLK>
__global__ void __launch_bounds__(BLK) k_conserved(Desc d, double* partials) {
  __shared__ double red[5][BLK];
  double acc[5] = {0, 0, 0, 0, 0};
  for (long long cell = (long long)blockIdx.x * BLK + threadIdx.x; cell < d.N;
       cell += (long long)gridDim.x * BLK) {
    if (d.mask != nullptr && d.mask[cell] != MASK_FLUID) continue;
    Nbr nb;
    if constexpr (ODD) nb = Nbr(d, coord_of(d, cell));
    const Raw r = gather_raw<ODD, P>(d, cell, nb);
    acc[0] += r.rho;
    acc[1] += r.jx;
    acc[2] += r.jy;
    acc[3] += r.jz;
    acc[4] += 0.5 * r.e2;
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

// Library reciprocals and CUDA's IEEE divisions side by side (diagnostic).
static __global__ void k_selftest_rcp(const double* x, double* y, double* ref, float* y32,
                                      float* ref32, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    y[i] = rcp64(x[i]);
    ref[i] = 1.0 / x[i];
    const float xf = (float)x[i];
    y32[i] = rcp32(xf);
    ref32[i] = 1.0f / xf;
  }
}

// Library exponential and CUDA's exp side by side (diagnostic).
static __global__ void k_selftest_exp(const double* x, double* y, double* ref, long long n) {
  load_exp_table();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    y[i] = exp_tang(x[i]);
    ref[i] = exp(x[i]);
  }
}

// FP64 FMA throughput probe: 8 independent chains per thread (diagnostic).
static __global__ void k_selftest_dfma(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x * 1e-9, x1 = x0 + 1e-9, x2 = x0 + 2e-9, x3 = x0 + 3e-9;
  double x4 = x0 + 4e-9, x5 = x0 + 5e-9, x6 = x0 + 6e-9, x7 = x0 + 7e-9;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

static __global__ void k_sum_partials(const double* partials, int nblocks, double* out5) {
  const int k = threadIdx.x;
  if (k >= 5) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += partials[b * 5 + k];
  out5[k] = s;
}

}  // namespace lbm39
