// cell.cuh -- per-cell arithmetic of the 13-moment DDF step (FP64).
//
// Every function runs in one thread for one cell.  Per-cell arrays that do
// not fit in registers live in shared memory with a stride of the block size
// (WS), so a warp touches 32 consecutive doubles and hits no bank conflict.
#pragma once
#include <cmath>

#include "d3q39.cuh"

namespace lbm39 {

// Strided per-thread view of a shared-memory array.
template <int BLK>
struct WS {
  double* p;
  __device__ __forceinline__ double& operator[](int k) const { return p[k * BLK]; }
  __device__ __forceinline__ WS at(int k) const { return WS{p + k * BLK}; }
};

// Per-thread workspace layout (units of BLK doubles).
constexpr int WS_F = 0;         // f populations (39)
constexpr int WS_G = 39;        // g populations (39)
constexpr int WS_E = 78;        // normalised equilibrium F_i (39)
constexpr int WS_LAM = 117;     // multipliers (13)
constexpr int WS_M = 130;       // normalised targets (13)
constexpr int WS_DOUBLES = 143;

// Lattice-wide constants of one run.
struct Phys {
  double tau;       // BGK relaxation time (tau_f = tau_g)
  double cg;        // 2 C_v - D (Eq. discrete-equilibrium-poly)
  double inv_2cv;   // 1 / (2 C_v)
  double tol;       // Newton tolerance on max_k |G_k| / rho
  int maxit;        // Newton updates allowed
  int min_upd;      // updates taken even from a converged warm start
  int kn_sensor;    // Eq. (alpha) on/off
};

// Targets of Eq. (13constraints) divided by rho:
// [1, u, u_a u_b + T delta_ab (xx,yy,zz,xy,xz,yz), u_a (u^2 + (D+2) T)].
// The contracted third moment is that of the Maxwellian, rho u_a (u^2 + 5T).
template <int BLK>
__device__ __forceinline__ void targets(double ux, double uy, double uz, double T, WS<BLK> m) {
  const double u2 = ux * ux + uy * uy + uz * uz;
  const double h = u2 + (D + 2) * T;
  m[0] = 1.0;
  m[1] = ux; m[2] = uy; m[3] = uz;
  m[4] = ux * ux + T; m[5] = uy * uy + T; m[6] = uz * uz + T;
  m[7] = ux * uy; m[8] = ux * uz; m[9] = uy * uz;
  m[10] = ux * h; m[11] = uy * h; m[12] = uz * h;
}

// F_i = exp(sum_k lam_k phi_k(xi_i)) (Eq. discrete-equilibrium / rho) into F,
// and the constraint residual G_k = sum_i F_i phi_k(xi_i) - m_k (Eq. constraints).
template <int BLK>
__device__ __forceinline__ void eval_equilibrium(const double (&l)[NM], WS<BLK> F, WS<BLK> m,
                                                 double (&G)[NM]) {
  double s[NM];
#pragma unroll
  for (int k = 0; k < NM; ++k) s[k] = 0.0;
  static_for<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    double e = l[0];
    static_for<1, NM>([&](auto K) {
      constexpr int k = decltype(K)::value;
      constexpr int c = phi(k, i);
      if constexpr (c == 1) e += l[k];
      else if constexpr (c == -1) e -= l[k];
      else if constexpr (c != 0) e = fma((double)c, l[k], e);
    });
    const double Fi = exp(e);
    F[i] = Fi;
    static_for<0, NM>([&](auto K) {
      constexpr int k = decltype(K)::value;
      constexpr int c = phi(k, i);
      if constexpr (c == 1) s[k] += Fi;
      else if constexpr (c == -1) s[k] -= Fi;
      else if constexpr (c != 0) s[k] = fma((double)c, Fi, s[k]);
    });
  });
#pragma unroll
  for (int k = 0; k < NM; ++k) G[k] = s[k] - m[k];
}

__device__ __forceinline__ double max_abs(const double (&v)[NM]) {
  double r = 0.0;
#pragma unroll
  for (int k = 0; k < NM; ++k) {
    const double a = fabs(v[k]);
    r = (a <= r) ? r : a;  // NaN propagates
  }
  return r;
}

__device__ __forceinline__ double sum_sq(const double (&v)[NM]) {
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < NM; ++k) s = fma(v[k], v[k], s);
  return s;
}

// Jacobian J_kl = sum_i F_i phi_k phi_l (Sec. 5 step table), packed lower
// triangle, then in place LDL^T and the solve J x = b (b overwritten by x).
// Returns false if a pivot is not positive (J not numerically SPD).
template <int BLK>
__device__ __forceinline__ bool jacobian_solve(WS<BLK> F, double (&b)[NM]) {
  double J[NTRI];
#pragma unroll
  for (int t = 0; t < NTRI; ++t) J[t] = 0.0;
  static_for<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const double Fi = F[i];
    static_for<0, NM>([&](auto K) {
      constexpr int k = decltype(K)::value;
      static_for<0, k + 1>([&](auto L) {
        constexpr int l = decltype(L)::value;
        constexpr int c = phi(k, i) * phi(l, i);
        if constexpr (c == 1) J[tri(k, l)] += Fi;
        else if constexpr (c == -1) J[tri(k, l)] -= Fi;
        else if constexpr (c != 0) J[tri(k, l)] = fma((double)c, Fi, J[tri(k, l)]);
      });
    });
  });
  bool ok = true;
  // LDL^T: diagonal d_j on J[tri(j,j)], unit-lower L below it.
  static_for<0, NM>([&](auto JJ) {
    constexpr int j = decltype(JJ)::value;
    double v[NM];
    static_for<0, j>([&](auto K) {
      constexpr int k = decltype(K)::value;
      v[k] = J[tri(j, k)] * J[tri(k, k)];
    });
    double dj = J[tri(j, j)];
    static_for<0, j>([&](auto K) {
      constexpr int k = decltype(K)::value;
      dj = fma(-J[tri(j, k)], v[k], dj);
    });
    ok = ok && (dj > 0.0);
    J[tri(j, j)] = dj;
    const double rj = 1.0 / dj;
    static_for<j + 1, NM>([&](auto II) {
      constexpr int i = decltype(II)::value;
      double a = J[tri(i, j)];
      static_for<0, j>([&](auto K) {
        constexpr int k = decltype(K)::value;
        a = fma(-J[tri(i, k)], v[k], a);
      });
      J[tri(i, j)] = a * rj;
    });
  });
  // L y = b
  static_for<1, NM>([&](auto II) {
    constexpr int i = decltype(II)::value;
    double a = b[i];
    static_for<0, i>([&](auto K) {
      constexpr int k = decltype(K)::value;
      a = fma(-J[tri(i, k)], b[k], a);
    });
    b[i] = a;
  });
  // D z = y
#pragma unroll
  for (int i = 0; i < NM; ++i) b[i] = b[i] / J[tri(i, i)];
  // L^T x = z
  static_for<0, NM - 1>([&](auto II) {
    constexpr int i = NM - 2 - decltype(II)::value;
    double a = b[i];
    static_for<i + 1, NM>([&](auto K) {
      constexpr int k = decltype(K)::value;
      a = fma(-J[tri(k, i)], b[k], a);
    });
    b[i] = a;
  });
  return ok;
}

constexpr int LS_MAX = 30;

struct NewtonResult {
  int n_upd;
  int failed;
};

// Newton-Raphson for the 13 multipliers (Sec. 3, Sec. 5 step table), from the
// multipliers in `lam` (warm start or Gaussian cold start).  Reading of the
// stopping rule: at least min_upd updates; stop when max|G| < tol, except
// that a solve landing in [tol/100, tol) takes one more full (polishing)
// step; while max|G| >= tol the step is halved until ||G||_2 decreases.
// On return F holds exp(Phi lam) at the returned lam.
template <int BLK>
__device__ NewtonResult newton(WS<BLK> lam, WS<BLK> F, WS<BLK> m, const Phys& ph, int maxit) {
  double l0[NM], G[NM];
#pragma unroll
  for (int k = 0; k < NM; ++k) l0[k] = lam[k];
  eval_equilibrium<BLK>(l0, F, m, G);
  int n = 0, failed = 0;
  bool polished = false;
  for (;;) {
    const double r = max_abs(G);
    if (n >= ph.min_upd && r < ph.tol && (r < 1e-2 * ph.tol || polished)) break;
    if (n >= maxit) { failed = 1; break; }
    const double s0 = sum_sq(G);
    if (!jacobian_solve<BLK>(F, G)) { failed = 1; break; }  // G now holds delta
#pragma unroll
    for (int k = 0; k < NM; ++k) l0[k] = lam[k];
    polished = r < ph.tol;
    double lt[NM], Gt[NM];
    if (polished) {
#pragma unroll
      for (int k = 0; k < NM; ++k) lt[k] = l0[k] - G[k];
      eval_equilibrium<BLK>(lt, F, m, Gt);
    } else {
      double t = 1.0;
      bool ok = false;
      for (int ls = 0; ls <= LS_MAX; ++ls) {
#pragma unroll
        for (int k = 0; k < NM; ++k) lt[k] = fma(-t, G[k], l0[k]);
        eval_equilibrium<BLK>(lt, F, m, Gt);
        if (sum_sq(Gt) < s0) { ok = true; break; }
        t *= 0.5;
      }
      if (!ok) {  // keep the last accepted point
        eval_equilibrium<BLK>(l0, F, m, Gt);
        failed = 1;
        break;
      }
    }
#pragma unroll
    for (int k = 0; k < NM; ++k) { lam[k] = lt[k]; G[k] = Gt[k]; }
    ++n;
  }
  return NewtonResult{n, failed};
}

// Gaussian cold start (reading): lam_1 = u/T, diagonal lam_2 = -1/(2T), the rest 0,
// lam_0 normalising sum_i F_i = 1.
template <int BLK>
__device__ __forceinline__ void gaussian_guess(double ux, double uy, double uz, double T,
                                               WS<BLK> lam) {
  const double it = 1.0 / T;
  double l[NM];
#pragma unroll
  for (int k = 0; k < NM; ++k) l[k] = 0.0;
  l[1] = ux * it; l[2] = uy * it; l[3] = uz * it;
  l[4] = l[5] = l[6] = -0.5 * it;
  double s = 0.0;
  static_for<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int cx = CX[i], cy = CY[i], cz = CZ[i], cc = c2(i);
    s += exp(l[1] * cx + l[2] * cy + l[3] * cz + l[4] * cc);
  });
  l[0] = -log(s);
#pragma unroll
  for (int k = 0; k < NM; ++k) lam[k] = l[k];
}

// alpha(eps) of Eq. (alpha).
__device__ __forceinline__ double alpha_of(double eps, double tau) {
  return eps < 1e-2 ? 1.0 : eps < 1e-1 ? 1.05 : eps < 1.0 ? 1.35 : 1.0 / tau;
}
__device__ __forceinline__ int alpha_branch(double eps) {
  return eps < 1e-2 ? 0 : eps < 1e-1 ? 1 : eps < 1.0 ? 2 : 3;
}

struct CellStats {
  int n_upd;
  int failed;
  int branch;
};

// One fluid-cell collision in FP64 (Sec. 3): f, g (post-streaming) in the
// workspace -> moments -> targets -> Newton (warm start in lam) -> f^eq,
// g^eq = (2C_v - D) T f^eq -> eps (f only) -> tau_eff = tau alpha(eps) ->
// BGK on f and g, written back into the workspace.
template <int BLK>
__device__ CellStats collide_fp64(WS<BLK> w, const Phys& ph) {
  WS<BLK> f = w.at(WS_F), g = w.at(WS_G), F = w.at(WS_E), lam = w.at(WS_LAM), m = w.at(WS_M);
  double rho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0, e2 = 0.0;
  static_for<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const double fi = f[i];
    rho += fi;
    constexpr int cx = CX[i], cy = CY[i], cz = CZ[i], cc = c2(i);
    if constexpr (cx != 0) jx = fma((double)cx, fi, jx);
    if constexpr (cy != 0) jy = fma((double)cy, fi, jy);
    if constexpr (cz != 0) jz = fma((double)cz, fi, jz);
    if constexpr (cc != 0) e2 = fma((double)cc, fi, e2);
    e2 += g[i];
  });
  const double ir = 1.0 / rho;
  const double ux = jx * ir, uy = jy * ir, uz = jz * ir;
  const double T = (e2 - rho * (ux * ux + uy * uy + uz * uz)) * ph.inv_2cv * ir;
  targets<BLK>(ux, uy, uz, T, m);
  const NewtonResult nr = newton<BLK>(lam, F, m, ph, ph.maxit);
  double eps = 0.0;
  static_for<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const double feq = rho * F[i];
    eps += fabs(f[i] - feq) / feq;
  });
  eps *= (1.0 / Q);
  const double alpha = ph.kn_sensor ? alpha_of(eps, ph.tau) : 1.0;
  const double omega = 1.0 / (ph.tau * alpha);
  const double cgr = ph.cg * T * rho;
  static_for<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const double Fi = F[i];
    const double fi = f[i], gi = g[i];
    f[i] = fi - omega * (fi - rho * Fi);
    g[i] = gi - omega * (gi - cgr * Fi);
  });
  return CellStats{nr.n_upd, nr.failed, alpha_branch(eps)};
}

}  // namespace lbm39
