// cell.cuh -- per-cell arithmetic of the 13-moment DDF step.
//
// Every function runs in one thread for one cell.  Per-cell arrays that do
// not fit in registers live in shared memory with a stride of the block size
// (WS), so a warp touches 32 consecutive doubles and hits no bank conflict.
//
// The GB300 issues FP64 at about 1/64 of the FP32 rate, so the FP64 step is
// bound by its FP64 operation count.  The sums over the 39 velocities come
// from gen_d3q39.py (sign-orbit butterflies: the same sums, reorganised), the
// exponential is exp_tang (9 FP64 operations), and the Knudsen sensor is
// screened in FP32 and recomputed in FP64 only near a threshold of Eq. (alpha),
// so alpha is the one an FP64 evaluation gives.
#pragma once
#include <cmath>

#include "d3q39.cuh"
#include "d3q39_gen.cuh"
#include "expd.cuh"

namespace lbm39 {

// Strided per-thread view of a shared-memory array.
template <class V, int BLK>
struct WSV {
  V* p;
  __device__ __forceinline__ V& operator[](int k) const { return p[k * BLK]; }
  __device__ __forceinline__ WSV at(int k) const { return WSV{p + k * BLK}; }
};
template <int BLK>
using WS = WSV<double, BLK>;

// Per-thread workspace layout (units of BLK doubles).
constexpr int WS_E = 0;         // normalised equilibrium F_i (39)
constexpr int WS_LAM = 39;      // multipliers (13)
constexpr int WS_M = 52;        // normalised targets (13)
constexpr int WS_DL = 65;       // Newton direction (13)
constexpr int WS_DOUBLES = 78;

// Lattice-wide constants of one run.
struct Phys {
  double tau;       // BGK relaxation time (tau_f = tau_g)
  double cg;        // 2 C_v - D (Eq. discrete-equilibrium-poly)
  double inv_2cv;   // 1 / (2 C_v)
  double tol;       // Newton tolerance on max_k |G_k| / rho
  int maxit;        // Newton updates allowed
  int min_upd;      // updates taken even from a converged warm start
  int kn_sensor;    // Eq. (alpha) on/off
  double omega[4];  // 1 / (tau alpha) for the four branches of Eq. (alpha) (1/tau without
                    // the sensor), formed on the host with IEEE division
  int pr_adjust;    // Prandtl-number adjustment on (Pr != 1)
  double domega[4]; // per branch: 1/tau_eff - 1/tau2, tau2 = 1/2 + (tau_eff - 1/2)/Pr
};

// Reciprocals without the IEEE division sequence.
// rcp32: the PTX instruction rcp.approx.ftz.f32 (at most 1 ulp, i.e. relative
// error <= 2^-23, subnormals flushed to zero).
__device__ __forceinline__ float rcp32(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// rcp64: 1/d for normal d by Newton's method for the root of 1/r - d,
// r <- r + r (1 - d r), each step squaring the relative error, two steps from
// the hardware estimate rcp.approx.ftz.f64.  Within 2 ulp of 1/d (tested
// against CUDA's division through lbm39_selftest_rcp).
__device__ __forceinline__ double rcp64(double d) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
  r = fma(r, fma(-d, r, 1.0), r);
  return fma(r, fma(-d, r, 1.0), r);
}

template <class T>
__device__ __forceinline__ T recip(T x) {
  if constexpr (sizeof(T) == 8) return rcp64(x);
  else return rcp32(x);
}

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

// Float view of a double by integer operations (truncated to 23 mantissa bits):
// relative error below 2^-23 for |x| in float's normal range, 0 below it.
__device__ __forceinline__ float trunc_float(double x) {
  const int hi = __double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const int e = ((hi >> 20) & 0x7ff) - 1023 + 127;
  if (e >= 255) return __double2float_rn(x);  // out of range, inf, NaN
  const unsigned bits = ((unsigned)hi & 0x80000000u) | ((unsigned)e << 23) |
                        (((unsigned)hi & 0xfffffu) << 3) | (lo >> 29);
  return e > 0 ? __uint_as_float(bits) : 0.0f;
}

// The same view in three integer operations for a double whose exponent E
// (biased, 11 bits) gives a normal float (897 <= E <= 1150; callers check E
// with exp_field): the funnel shift leaves E mod 512 above the top 23
// mantissa bits, and subtracting 384 in that 9-bit field leaves E - 896.
__device__ __forceinline__ float view_float(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned m = __funnelshift_l(lo, hi, 3);
  return __uint_as_float((m - (384u << 23)) | (hi & 0x80000000u));
}

// Biased exponent field of a double (bits 52..62 in place, as an int).
__device__ __forceinline__ int exp_field(double x) { return __double2hiint(x) & 0x7ff00000; }

// exp of the 39 exponents parked in F (stride BLK), by CUDA's exp: the rare
// path for arguments outside exp_tang_core's range.
template <int BLK>
__device__ __noinline__ void exp_all_slow(double* Fp) {
  for (int i = 0; i < Q; ++i) Fp[i * BLK] = exp(Fp[i * BLK]);
}

// F_i = exp(sum_k lam_k phi_k(xi_i)) (Eq. discrete-equilibrium / rho) into F,
// and the constraint residual G_k = sum_i F_i phi_k(xi_i) - m_k (Eq. constraints).
// The evaluation point is lam - t dl (t = 0: lam itself, dl not read); dl holds
// the direction of the system's multipliers (Sys<D2>: all 13, or the nine
// z-even ones, whose G this returns).
// from_F: F already holds exp(Phi lam) (kept from the previous step), so only
// the moments are formed -- the same numbers, bit for bit, as evaluating again.
// D2: z-mirrored velocities share their exponential.
template <int BLK, bool D2 = false>
__device__ __forceinline__ void eval_equilibrium(WS<BLK> lam, WS<BLK> dl, double t, WS<BLK> F,
                                                 WS<BLK> m, double (&G)[Sys<D2>::N],
                                                 bool from_F) {
  using S = Sys<D2>;
  if (!from_F) {
    double l[NM], x[Q];
#pragma unroll
    for (int k = 0; k < NM; ++k) l[k] = lam[k];
    if (t != 0.0) {
#pragma unroll
      for (int k = 0; k < S::N; ++k) l[S::idx(k)] = fma(-t, dl[k], lam[S::idx(k)]);
    }
    if constexpr (D2) gen::exponents2d(l, x);
    else gen::exponents(l, x);
    int wide = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      wide |= exp_out_of_range(x[i]);
      F[i] = x[i];
    }
    if (wide) {  // |e| >= 512, inf or NaN somewhere: CUDA's exp for all 39
      exp_all_slow<BLK>(F.p);
    } else {
      // one exponential at a time from the workspace: a single copy of its code
      // (the FP64 pipe's issue rate, not the chain's latency, paces it); D2: once
      // per z-mirror pair, then copied
#pragma unroll 1
      for (int i = 0; i < Q; ++i)
        if (!D2 || ((kZOwn >> i) & 1ull)) F[i] = exp_tang_core(F[i]);
      if constexpr (D2) {
        static_for<0, Q>([&](auto I) {
          constexpr int i = decltype(I)::value;
          if constexpr (zmirror(i) < i) F[i] = F[zmirror(i)];
        });
      }
    }
  }
  double s[S::N];
  if constexpr (D2) gen::moments_s2d<double>(F, s);
  else gen::moments_s<double>(F, s);
#pragma unroll
  for (int k = 0; k < S::N; ++k) G[k] = s[k] - m[S::idx(k)];
}

template <class T, int N>
__device__ __forceinline__ T max_abs(const T (&v)[N]) {
  T r = T(0);
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const T a = fabs(v[k]);
    r = (a <= r) ? r : a;  // NaN propagates
  }
  return r;
}

template <int N>
__device__ __forceinline__ double sum_sq(const double (&v)[N]) {
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < N; ++k) s = fma(v[k], v[k], s);
  return s;
}

// In-place LDL^T of a packed symmetric N x N J: unit-lower L below a diagonal
// D, with rd the reciprocals of D's entries.  False if a pivot is not positive
// (J not numerically SPD).  Right-looking elimination: pivot k scales its column
// once (L_ik = a_ik / d_k) and updates the trailing matrix with a_ij -= L_ik a_jk,
// so each multiplier is one product and every other operation a fused
// multiply-add (in FP64 the FP64 pipe bounds the step), and the updates of a
// column are independent of one another (short dependency chains for the FP32
// factorisations of the single-precision direction).
template <class T, int N = NM>
__device__ __forceinline__ bool ldlt_factor(T (&J)[N * (N + 1) / 2], T (&rd)[N]) {
  bool ok = true;
  static_for<0, N>([&](auto KK) {
    constexpr int k = decltype(KK)::value;
    const T dk = J[tri(k, k)];
    ok = ok && (dk > T(0));
    rd[k] = recip(dk);
    T w[N];  // column k below the pivot, unscaled
    static_for<k + 1, N>([&](auto II) {
      constexpr int i = decltype(II)::value;
      w[i] = J[tri(i, k)];
      J[tri(i, k)] = w[i] * rd[k];
    });
    static_for<k + 1, N>([&](auto II) {
      constexpr int i = decltype(II)::value;
      static_for<k + 1, i + 1>([&](auto JJ) {
        constexpr int j = decltype(JJ)::value;
        J[tri(i, j)] = fma(-J[tri(i, k)], w[j], J[tri(i, j)]);
      });
    });
  });
  return ok;
}

// Solve J x = b with the factor of ldlt_factor (b overwritten by x).
template <class T, int N = NM>
__device__ __forceinline__ void ldlt_apply(const T (&J)[N * (N + 1) / 2], const T (&rd)[N],
                                           T (&b)[N]) {
  static_for<1, N>([&](auto II) {  // L y = b
    constexpr int i = decltype(II)::value;
    T a = b[i];
    static_for<0, i>([&](auto K) {
      constexpr int k = decltype(K)::value;
      a = fma(-J[tri(i, k)], b[k], a);
    });
    b[i] = a;
  });
#pragma unroll
  for (int i = 0; i < N; ++i) b[i] *= rd[i];  // D z = y
  static_for<0, N - 1>([&](auto II) {  // L^T x = z
    constexpr int i = N - 2 - decltype(II)::value;
    T a = b[i];
    static_for<i + 1, N>([&](auto K) {
      constexpr int k = decltype(K)::value;
      a = fma(-J[tri(k, i)], b[k], a);
    });
    b[i] = a;
  });
}

// Position of L_ik (i > k, k < KS) when the first KS columns of L are parked in
// a workspace array column after column.
template <int N>
constexpr int parked(int i, int k) {
  int off = 0;
  for (int c = 0; c < k; ++c) off += N - 1 - c;
  return off + (i - k - 1);
}

// ldlt_apply with the first KS columns of L read from the workspace array P
// (parked there by the caller), the others from J.
template <int N, int KS, int BLK>
__device__ __forceinline__ void ldlt_apply_parked(const double (&J)[N * (N + 1) / 2],
                                                  const double (&rd)[N], WS<BLK> P,
                                                  double (&b)[N]) {
  static_for<1, N>([&](auto II) {  // L y = b
    constexpr int i = decltype(II)::value;
    double a = b[i];
    static_for<0, i>([&](auto K) {
      constexpr int k = decltype(K)::value;
      const double l = k < KS ? P[parked<N>(i, k)] : J[tri(i, k)];
      a = fma(-l, b[k], a);
    });
    b[i] = a;
  });
#pragma unroll
  for (int i = 0; i < N; ++i) b[i] *= rd[i];  // D z = y
  static_for<0, N - 1>([&](auto II) {  // L^T x = z
    constexpr int i = N - 2 - decltype(II)::value;
    double a = b[i];
    static_for<i + 1, N>([&](auto K) {
      constexpr int k = decltype(K)::value;
      const double l = i < KS ? P[parked<N>(k, i)] : J[tri(k, i)];
      a = fma(-l, b[k], a);
    });
    b[i] = a;
  });
}

// In-place LDL^T of a packed symmetric N x N J and the solve J x = b (b
// overwritten by x).  False if a pivot is not positive.
template <class T, int N = NM>
__device__ __forceinline__ bool ldlt_solve(T (&J)[N * (N + 1) / 2], T (&b)[N]) {
  T rd[N];
  const bool ok = ldlt_factor<T, N>(J, rd);
  ldlt_apply<T, N>(J, rd, b);
  return ok;
}

// Single-precision direction (the precision form's Newton steps and the
// single-precision start): J = sum_i F_i phi phi^T from the float equilibrium
// at Fp (Q values), J d = b by the float LDL^T, b at bp (the system's N values,
// overwritten by d).  False if a pivot is not positive.  Not inlined: its one
// copy serves both callers, which keeps the step kernel's code (and its
// instruction-cache footprint) small; the arrays pass through the stack.
template <bool D2>
__device__ __noinline__ bool dir32(const float* __restrict__ Fp, float* __restrict__ bp) {
  constexpr int N = Sys<D2>::N;
  float Ff[Q], J[N * (N + 1) / 2], s[N], b[N];
#pragma unroll
  for (int i = 0; i < Q; ++i) Ff[i] = Fp[i];
  if constexpr (D2) gen::moments2d<float>(Ff, s, J);
  else gen::moments<float>(Ff, s, J);
#pragma unroll
  for (int k = 0; k < N; ++k) b[k] = bp[k];
  const bool ok = ldlt_solve<float, N>(J, b);
#pragma unroll
  for (int k = 0; k < N; ++k) bp[k] = b[k];
  return ok;
}

// Newton direction: J = sum_i F_i phi phi^T (Sec. 5 step table), J delta = b,
// b and delta in dl.  FP64 path: J and LDL^T in FP64.  Precision form: in
// FP32 (dir32; the residual and the update stay FP64, so the iteration still
// converges to the FP64 root).
template <int BLK, bool MIXED, bool D2 = false>
__device__ __forceinline__ bool newton_direction(WS<BLK> F, WS<BLK> dl) {
  constexpr int N = Sys<D2>::N;
  if constexpr (!MIXED) {
    double J[N * (N + 1) / 2], s[N], b[N], rd[N];
    if constexpr (D2) gen::moments2d<double>(F, s, J);
    else gen::moments<double>(F, s, J);
    const bool ok = ldlt_factor<double, N>(J, rd);
    if constexpr (D2) {
#pragma unroll
      for (int k = 0; k < N; ++k) b[k] = dl[k];  // the right-hand side, once J is factored
      ldlt_apply<double, N>(J, rd, b);
    } else {
      // The 13x13 solve needs L, D and b at once (more than the registers hold): the
      // first three columns of L (33 values) wait in F's workspace slots, which the next
      // evaluation overwrites before anything reads them.
      constexpr int KS = 3;
      static_for<0, KS>([&](auto K) {
        constexpr int k = decltype(K)::value;
        static_for<k + 1, N>([&](auto II) {
          constexpr int i = decltype(II)::value;
          F[parked<N>(i, k)] = J[tri(i, k)];
        });
      });
#pragma unroll
      for (int k = 0; k < N; ++k) b[k] = dl[k];
      ldlt_apply_parked<N, KS, BLK>(J, rd, F, b);
    }
#pragma unroll
    for (int k = 0; k < N; ++k) dl[k] = b[k];
    return ok;
  } else {
    float Ff[Q], bf[N];
#pragma unroll
    for (int i = 0; i < Q; ++i) Ff[i] = trunc_float(F[i]);
#pragma unroll
    for (int k = 0; k < N; ++k) bf[k] = trunc_float(dl[k]);
    const bool ok = dir32<D2>(Ff, bf);
#pragma unroll
    for (int k = 0; k < N; ++k) dl[k] = (double)bf[k];
    return ok;
  }
}

constexpr int LS_MAX = 30;

struct NewtonResult {
  int n_upd;
  int failed;
};

// Newton-Raphson for the multipliers (Sec. 3, Sec. 5 step table; all 13, or
// with D2 the nine z-even ones, the others staying exactly zero), from the
// multipliers in `lam` (warm start or Gaussian cold start).  Reading of the
// stopping rule: stop when max|G| < tol, after at least min_upd updates,
// except that a solve landing in [tol/100, tol) takes one more full
// (polishing) step; while max|G| >= tol the step is halved until ||G||_2
// decreases.  On return F holds exp(Phi lam) at the returned lam.
// One evaluation site and one direction site keep the unrolled code small;
// trial point and direction live in the workspace (w: the cell's workspace).
// cached: F already holds exp(Phi lam) for the starting lam (the previous
// step's last evaluation, kept per cell), so the first evaluation skips the
// exponentials.
template <int BLK, bool MIXED, bool D2 = false>
__device__ NewtonResult newton(WS<BLK> w, const Phys& ph, int maxit, bool cached) {
  using S = Sys<D2>;
  WS<BLK> lam = w.at(WS_LAM), F = w.at(WS_E), m = w.at(WS_M), dl = w.at(WS_DL);
  int n = 0, failed = 0, ls = 0;
  bool first = true, polished = false, restore = false;
  double t = 0.0, s0 = 0.0;  // trial point lam - t dl
  for (;;) {
    double G[S::N];
    eval_equilibrium<BLK, D2>(lam, dl, t, F, m, G, first && cached);
    if (restore) break;  // F is back at the last accepted lam after a failed line search
    if (!first && !polished && !(sum_sq(G) < s0)) {  // reject: halve the step
      if (++ls > LS_MAX) {
        failed = 1;
        restore = true;
        t = 0.0;
        continue;
      }
      t *= 0.5;
      continue;
    }
    // accept the trial point
    if (t != 0.0) {
#pragma unroll
      for (int k = 0; k < S::N; ++k) lam[S::idx(k)] = fma(-t, dl[k], lam[S::idx(k)]);
    }
    if (!first) ++n;
    first = false;
    const double r = max_abs(G);
    if (n >= ph.min_upd && r < ph.tol && (r < 1e-2 * ph.tol || polished)) break;
    if (n >= maxit) { failed = 1; break; }
    s0 = sum_sq(G);
#pragma unroll
    for (int k = 0; k < S::N; ++k) dl[k] = G[k];
    if (!newton_direction<BLK, MIXED, D2>(F, dl)) { failed = 1; break; }
    polished = r < ph.tol;
    t = 1.0;
    ls = 0;
  }
  return NewtonResult{n, failed};
}

// Single-precision start of a solve (root finder 3, and the precision form's
// solver).  From a warm start the first Newton steps need the residual only to a
// few digits, and float arithmetic issues at 64 times the FP64 rate here.  From
// F~ = F in float (F: the cached exp(Phi lam)), Newton steps in float: the float
// residual G of F~ (the generated sums), J d = G (dir32), and the trial
// equilibrium F~_i exp(-phi(xi_i) . d) with its residual; while max|G| >=
// START32_THETA, at most START32_MAXIT times, and a step is kept only if it lowers
// max|G| (else the phase ends).  Then lam -= (the sum of the kept d) in FP64, and
// the FP64-residual Newton finishes the solve from there, so the equilibrium is
// the one every root finder reaches.  Returns the number of steps kept (0: lam
// and the cached F untouched).
constexpr float START32_THETA = 1e-4f;
constexpr int START32_MAXIT = 4;

template <int BLK, bool D2 = false>
__device__ __forceinline__ int start32(WS<BLK> w) {
  using S = Sys<D2>;
  constexpr int N = S::N;
  WS<BLK> lam = w.at(WS_LAM), F = w.at(WS_E), m = w.at(WS_M);
  float Ff[Q], G[N], dsum[N];
#pragma unroll
  for (int i = 0; i < Q; ++i) Ff[i] = trunc_float(F[i]);
  {
    float s[N];
    if constexpr (D2) gen::moments_s2d<float>(Ff, s);
    else gen::moments_s<float>(Ff, s);
#pragma unroll
    for (int k = 0; k < N; ++k) {
      G[k] = s[k] - trunc_float(m[S::idx(k)]);
      dsum[k] = 0.0f;
    }
  }
  float r = max_abs(G);
  int n = 0;
  while (n < START32_MAXIT && r >= START32_THETA) {  // false for a NaN residual
    float d[N];
#pragma unroll
    for (int k = 0; k < N; ++k) d[k] = G[k];
    if (!dir32<D2>(Ff, d)) break;
    float l[NM], x[Q];  // -d at the system's places of the 13, and its exponents
#pragma unroll
    for (int k = 0; k < NM; ++k) l[k] = 0.0f;
#pragma unroll
    for (int k = 0; k < N; ++k) l[S::idx(k)] = -d[k];
    if constexpr (D2) gen::exponents2d<float>(l, x);
    else gen::exponents<float>(l, x);
#pragma unroll
    for (int i = 0; i < Q; ++i) x[i] = Ff[i] * expf(x[i]);
    float s[N];
    if constexpr (D2) gen::moments_s2d<float>(x, s);
    else gen::moments_s<float>(x, s);
#pragma unroll
    for (int k = 0; k < N; ++k) s[k] -= trunc_float(m[S::idx(k)]);
    const float rt = max_abs(s);
    if (!(rt < r)) break;
#pragma unroll
    for (int i = 0; i < Q; ++i) Ff[i] = x[i];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      G[k] = s[k];
      dsum[k] += d[k];
    }
    r = rt;
    ++n;
  }
  if (n > 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) lam[S::idx(k)] -= (double)dsum[k];
  }
  return n;
}

// Chord-Newton hybrid for the same equations (a second root finder; the
// paper's outlook names other root finders).  Same stopping rule, polishing
// step, budget, line search and failure rule as newton(); the direction reuses
// the LDL^T factor of the last Jacobian formed in this solve (a chord step)
// while the previous accepted step reduced max|G| by at least CHORD_RHO, and
// otherwise forms and factors J at the current point (a Newton step).  A chord
// step that does not reduce ||G||_2 is not halved: the solve goes back to the
// current point and takes a Newton step from there.  The factor (FP64) lives
// across the evaluations of the solve.
constexpr double CHORD_RHO = 1e-3;

template <int BLK, bool D2 = false>
__device__ NewtonResult newton_chord(WS<BLK> w, const Phys& ph, int maxit, bool cached) {
  using S = Sys<D2>;
  constexpr int N = S::N;
  WS<BLK> lam = w.at(WS_LAM), F = w.at(WS_E), m = w.at(WS_M), dl = w.at(WS_DL);
  int n = 0, failed = 0, ls = 0;
  bool first = true, polished = false, restore = false, refresh = false, chord = false;
  bool have_J = false;
  double t = 0.0, s0 = 0.0, r_prev = 0.0, r_dir = 0.0;
  double Jf[N * (N + 1) / 2], rd[N];
  for (;;) {
    double G[N];
    eval_equilibrium<BLK, D2>(lam, dl, t, F, m, G, first && cached);
    if (restore) break;  // F is back at the last accepted lam after a failed line search
    if (refresh) {
      refresh = false;  // back at lam after a rejected chord step: a Newton step from here
    } else {
      if (!first && !polished && !(sum_sq(G) < s0)) {  // reject
        if (chord) {  // a chord step is not halved
          refresh = true;
          have_J = false;
          r_prev = 0.0;
          t = 0.0;
          continue;
        }
        if (++ls > LS_MAX) {
          failed = 1;
          restore = true;
          t = 0.0;
          continue;
        }
        t *= 0.5;
        continue;
      }
      // accept the trial point
      if (t != 0.0) {
#pragma unroll
        for (int k = 0; k < N; ++k) lam[S::idx(k)] = fma(-t, dl[k], lam[S::idx(k)]);
      }
      if (!first) {
        ++n;
        r_prev = r_dir;
      }
      first = false;
    }
    const double r = max_abs(G);
    if (n >= ph.min_upd && r < ph.tol && (r < 1e-2 * ph.tol || polished)) break;
    if (n >= maxit) { failed = 1; break; }
    s0 = sum_sq(G);
    chord = have_J && r_prev > 0.0 && r <= CHORD_RHO * r_prev;
    if (!chord) {
      double s[N];
      if constexpr (D2) gen::moments2d<double>(F, s, Jf);
      else gen::moments<double>(F, s, Jf);
      if (!ldlt_factor<double, N>(Jf, rd)) { failed = 1; break; }
      have_J = true;
    }
    double b[N];
#pragma unroll
    for (int k = 0; k < N; ++k) b[k] = G[k];
    ldlt_apply<double, N>(Jf, rd, b);
#pragma unroll
    for (int k = 0; k < N; ++k) dl[k] = b[k];
    polished = r < ph.tol;
    r_dir = r;
    t = 1.0;
    ls = 0;
  }
  return NewtonResult{n, failed};
}

// ---------------------------------------------------------------------------
// Fallback where the 13-moment equilibrium does not exist (reading: the paper
// does not say what a cell does when its constraint solve fails).  Outside the
// moment cone of the 39 velocities no positive distribution has the 13 target
// moments, and Newton cannot converge.  Such a cell relaxes instead to the
// maximum-entropy equilibrium under the five collision invariants [1, xi,
// |xi|^2] only, F_i = exp(mu_0 + mu.xi_i + mu_4 |xi_i|^2) with
// sum_i F_i [1, xi_i, |xi_i|^2] = [1, u, u^2 + D T]: it exists far beyond that
// cone and conserves mass, momentum and energy (g^eq = (2 C_v - D) T f^eq as
// for the full equilibrium).  Same damped Newton iteration and stopping rule
// as the full solve, from the Gaussian start.  The five multipliers enter the
// exponent as the embedding (mu_0, mu_x, mu_y, mu_z, mu_4, mu_4, mu_4, 0...) of
// the 13, so the evaluation uses the full solve's generated exponent and
// moment sums, and those 13 sums give the 5 x 5 Jacobian but for one entry,
// sum_i F_i |xi_i|^4.  A non-inlined function (one copy of this code).
constexpr int N5 = 5;
constexpr int FALLBACK_MAXIT = 50;
constexpr double FALLBACK_TOL = 1e-12;
// Failure policy (reading; the paper is silent).  After a fallback the cell
// keeps its five multipliers embedded in the 13: lam = (mu_0, mu_x, mu_y, mu_z,
// mu_4, mu_4, mu_4, 0, 0, 0, 0, 0, 0), whose exp(Phi lam) is the fallback
// equilibrium, and it is flagged "on the fallback".  The flag is stored in
// the multipliers themselves: lam_9 = -0 in the embedding (it changes no
// exponent).  A converged solve, or a fallback that fails too, clears it
// (lam_9 + 0 turns -0 into +0 and leaves any other value alone), so a solved
// state, even one at rest with the same shape, is never taken for one.  A
// flagged cell retries the full solve from the embedding with the full Newton
// budget on the time steps that are multiples of RETRY_PERIOD (from the
// embedding the solve takes 5-7 updates even well inside the cone, so a cell
// that has come back inside returns there), and on the other steps takes no
// update and goes straight to the fallback, which starts from the stored mu.
// The schedule depends on the time step alone.
constexpr int RETRY_PERIOD = 8;  // a power of two

// F = exp(phi5 . (mu - t dl)) (t = 0: mu itself), the 13 sums s_k = sum_i F_i
// phi_k(xi_i) at that point, and G = sum_i F_i phi5(xi_i) - m5 (phi5 = [1, xi,
// |xi|^2], so its sums are s_0..s_3 and s_4 + s_5 + s_6).
template <int BLK>
__device__ __forceinline__ void eval5(WS<BLK> mu, WS<BLK> dl, double t, WS<BLK> F,
                                      const double (&m5)[N5], double (&G)[N5],
                                      double (&s)[NM]) {
  double v[N5];
#pragma unroll
  for (int k = 0; k < N5; ++k) v[k] = t == 0.0 ? mu[k] : fma(-t, dl[k], mu[k]);
  const double l[NM] = {v[0], v[1], v[2], v[3], v[4], v[4], v[4], 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  double x[Q];
  gen::exponents(l, x);
  int wide = 0;
#pragma unroll
  for (int i = 0; i < Q; ++i) wide |= exp_out_of_range(x[i]);
  if (wide) {  // |e| >= 512, inf or NaN somewhere: CUDA's exp for all 39
#pragma unroll
    for (int i = 0; i < Q; ++i) F[i] = x[i];
    exp_all_slow<BLK>(F.p);
#pragma unroll
    for (int i = 0; i < Q; ++i) x[i] = F[i];
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      x[i] = exp_tang_core(x[i]);
      F[i] = x[i];
    }
  }
  gen::moments_s<double>(x, s);
  G[0] = s[0] - m5[0];
  G[1] = s[1] - m5[1];
  G[2] = s[2] - m5[2];
  G[3] = s[3] - m5[3];
  G[4] = ((s[4] + s[5]) + s[6]) - m5[4];
}

// Newton direction of the fallback: J = sum_i F_i phi5 phi5^T (symmetric
// positive definite) from the 13 sums s of the same F and sum_i F_i |xi_i|^4,
// J d = b by elimination without pivoting; false if a pivot is not positive.
template <int BLK>
__device__ __forceinline__ bool direction5(WS<BLK> F, const double (&s)[NM], double (&b)[N5]) {
  double q[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};  // sum of F_i over each |xi|^2 in {1,3,4,8,9}
  static_for<1, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int r = c2(i);
    constexpr int k = r == 1 ? 0 : r == 3 ? 1 : r == 4 ? 2 : r == 8 ? 3 : 4;
    q[k] += F[i];
  });
  const double e4 = fma(81.0, q[4], fma(64.0, q[3], fma(16.0, q[2], fma(9.0, q[1], q[0]))));
  const double e2 = (s[4] + s[5]) + s[6];
  double A[N5][N5] = {{s[0], s[1], s[2], s[3], e2},
                      {s[1], s[4], s[7], s[8], s[10]},
                      {s[2], s[7], s[5], s[9], s[11]},
                      {s[3], s[8], s[9], s[6], s[12]},
                      {e2, s[10], s[11], s[12], e4}};
  bool ok = true;
#pragma unroll
  for (int c = 0; c < N5; ++c) {
    ok = ok && (A[c][c] > 0.0);
    const double ip = 1.0 / A[c][c];
#pragma unroll
    for (int r = c + 1; r < N5; ++r) {
      const double f = A[r][c] * ip;
#pragma unroll
      for (int k = c; k < N5; ++k) A[r][k] = fma(-f, A[c][k], A[r][k]);
      b[r] = fma(-f, b[c], b[r]);
    }
  }
#pragma unroll
  for (int r = N5 - 1; r >= 0; --r) {
    double a = b[r];
#pragma unroll
    for (int k = r + 1; k < N5; ++k) a = fma(-A[r][k], b[k], a);
    b[r] = a / A[r][r];
  }
  return ok;
}

// True if the multipliers in the workspace have the fallback's embedded form.
template <int BLK>
__device__ __forceinline__ bool is_fallback_embedding(WS<BLK> lam) {
  unsigned long long rest = 0;
#pragma unroll
  for (int k = 7; k < NM; ++k)
    if (k != 9) rest |= (unsigned long long)__double_as_longlong(lam[k]);
  const long long a = __double_as_longlong(lam[4]), b = __double_as_longlong(lam[5]),
                  c = __double_as_longlong(lam[6]);
  return (unsigned long long)__double_as_longlong(lam[9]) == 0x8000000000000000ull &&
         rest == 0 && a == b && b == c;
}

// The fallback equilibrium into F for the cell whose 13 normalised targets
// are in the workspace (m: their u and second moments give the five targets),
// from the five multipliers warm[] (a stored embedding) or, with warm null, the
// Gaussian start; leaves mu in the first five m slots and overwrites the dl
// slots.  Returns 1 if its solve fails too (F then holds a partial iterate).
template <int BLK>
__device__ __noinline__ int fallback_equilibrium(WS<BLK> w, double T, const double* warm) {
  WS<BLK> F = w.at(WS_E), mu = w.at(WS_M), dl = w.at(WS_DL);
  const double m5[N5] = {1.0, mu[1], mu[2], mu[3], mu[4] + mu[5] + mu[6]};
  double G[N5], s[NM];
  if (warm) {
#pragma unroll
    for (int k = 0; k < N5; ++k) mu[k] = warm[k];
  } else {
    const double it = 1.0 / T;
    mu[0] = 0.0;
    mu[1] = m5[1] * it; mu[2] = m5[2] * it; mu[3] = m5[3] * it;
    mu[4] = -0.5 * it;
    eval5<BLK>(mu, dl, 0.0, F, m5, G, s);
    mu[0] = -log(s[0]);  // normalises sum_i F_i to 1
  }
  eval5<BLK>(mu, dl, 0.0, F, m5, G, s);
  int n = 0, ls = 0;
  bool polished = false, first = true;
  double t = 0.0, s0 = 0.0;
  for (;;) {
    if (!first) {
      eval5<BLK>(mu, dl, t, F, m5, G, s);
      double ss = 0.0;
#pragma unroll
      for (int k = 0; k < N5; ++k) ss = fma(G[k], G[k], ss);
      if (!polished && !(ss < s0)) {  // reject: halve the step
        if (++ls > LS_MAX) return 1;
        t *= 0.5;
        continue;
      }
#pragma unroll
      for (int k = 0; k < N5; ++k) mu[k] = fma(-t, dl[k], mu[k]);
      ++n;
    }
    first = false;
    double r = 0.0, ss = 0.0;
#pragma unroll
    for (int k = 0; k < N5; ++k) {
      const double a = fabs(G[k]);
      r = (a <= r) ? r : a;
      ss = fma(G[k], G[k], ss);
    }
    if (r < FALLBACK_TOL && (r < 1e-2 * FALLBACK_TOL || polished)) return 0;
    if (n >= FALLBACK_MAXIT) return 1;
    s0 = ss;
    double b[N5];
#pragma unroll
    for (int k = 0; k < N5; ++k) b[k] = G[k];
    if (!direction5<BLK>(F, s, b)) return 1;
#pragma unroll
    for (int k = 0; k < N5; ++k) dl[k] = b[k];
    polished = r < FALLBACK_TOL;
    t = 1.0;
    ls = 0;
  }
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
  double e[Q];
  gen::exponents(l, e);
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < Q; ++i) s += exp(e[i]);
  l[0] = -log(s);
#pragma unroll
  for (int k = 0; k < NM; ++k) lam[k] = l[k];
}

// Branch of alpha(eps) in Eq. (alpha): eps < 1e-2, < 1e-1, < 1, >= 1 (Phys::omega).
__device__ __forceinline__ int alpha_branch(double eps) {
  return eps < 1e-2 ? 0 : eps < 1e-1 ? 1 : eps < 1.0 ? 2 : 3;
}

// 1 / tau_eff of that branch (selects, so the table is not indexed at run time).
__device__ __forceinline__ double omega_of(const Phys& ph, int branch) {
  return branch == 0 ? ph.omega[0] : branch == 1 ? ph.omega[1] : branch == 2 ? ph.omega[2]
                                                                            : ph.omega[3];
}

// 1/tau_eff - 1/tau2 of that branch (Prandtl-number adjustment).
__device__ __forceinline__ double domega_of(const Phys& ph, int branch) {
  return branch == 0 ? ph.domega[0] : branch == 1 ? ph.domega[1] : branch == 2 ? ph.domega[2]
                                                                              : ph.domega[3];
}

// FP32 screen of s = 39 eps = sum_i |f_i - f^eq_i| / f^eq_i (Eq. DeltaAvg).  With
// u = 2^-24: each float view (f~, F~, rho~) is within 2u of its double, q = rho~ F~
// adds u, the difference u, rcp32 2u and the product u, so each term is within
// 7u + 11u t of t (using |f| / f^eq <= 1 + t); four interleaved partial sums of at
// most 10 terms add at most 11u s.  In all |s32 - s| <= u (273 + 22 s), i.e.
// 1.63e-5 + 1.31e-6 s, provided every view and q are normal floats: F_i, |f_i| in
// [2^-100, 2^100] (exponent fields within SCREEN_EMIN..SCREEN_EMAX) and rho~ in
// [2^-20, 2^20].  True when that fails, when s32 is not finite, or when s32 lies
// within 3e-5 + 3e-6 s32 (about twice the bound) of a threshold 39 * {1e-2, 1e-1, 1}:
// then the FP64 value decides the branch.
constexpr int SCREEN_EMIN = (1023 - 100) << 20, SCREEN_EMAX = (1023 + 100) << 20;

__device__ __forceinline__ bool screen_undecided(float s39, int emin, int emax, float rho32) {
  if (!(s39 < 1e30f) || emin < SCREEN_EMIN || emax > SCREEN_EMAX ||
      !(rho32 >= 0x1p-20f && rho32 <= 0x1p20f))
    return true;
  const float band = 3e-5f + 3e-6f * s39;
  return fabsf(s39 - 0.39f) <= band || fabsf(s39 - 3.9f) <= band || fabsf(s39 - 39.0f) <= band;
}

// The screen of the precision form, whose terms are |d_i| r_i with d_i = f~_i - rf_i
// the float difference of the stored deviation and the equilibrium's, rf_i =
// f^eq_i - f_ref_i rounded to the nearest float, and r_i = rcp32(rho~ F~_i).  With u = 2^-24: d_i is
// within u|d_i| of the exact difference, r_i within 7u of 1/f^eq_i (two float views 2u
// each, the product u, rcp32 2u), the product adds u, and four interleaved partial sums
// of at most 10 terms add at most 12u s: |s32 - s| <= 21u s32 to first order.  True when
// s32 is not finite (a view out of float's range makes r_i infinite) or lies within
// 2^-18 s32 (about twice the bound) of a threshold 39 * {1e-2, 1e-1, 1}.
__device__ __forceinline__ bool screen_undecided_dev(float s39) {
  if (!(s39 < 1e30f)) return true;
  const float band = 0x1p-18f * s39;
  return fabsf(s39 - 0.39f) <= band || fabsf(s39 - 3.9f) <= band || fabsf(s39 - 39.0f) <= band;
}

struct CellStats {
  int n_upd;
  int failed;
  int branch;
};

// Macroscopic variables (Sec. 3): rho, u and T from the total energy,
// sum f|xi|^2 + sum g = rho u^2 + 2 C_v rho T (E = u^2/2 + C_v T, Sec. 2).
struct Macro {
  double rho, ux, uy, uz, T;
};

__device__ __forceinline__ Macro macro_from_moments(double rho, double jx, double jy, double jz,
                                                    double e2, double inv_2cv) {
  const double ir = rcp64(rho);
  Macro M;
  M.rho = rho;
  M.ux = jx * ir; M.uy = jy * ir; M.uz = jz * ir;
  M.T = (e2 - rho * (M.ux * M.ux + M.uy * M.uy + M.uz * M.uz)) * inv_2cv * ir;
  return M;
}

}  // namespace lbm39
