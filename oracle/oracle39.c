/*
 * oracle39.c -- plain, slow FP64 CPU oracle of the 13-moment guided-equilibrium
 * double-distribution-function lattice Boltzmann step on D3Q39
 * (Latt, Coreixas, Beny, Parmigiani, "Efficient supersonic flows through
 * high-order guided equilibrium with lattice Boltzmann", arXiv:1910.13515).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference the CUDA path is
 * checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code, table or header with
 * the CUDA library; the product path never calls it.
 *
 * Every function follows the paper's algorithm in the paper's order, written
 * for a reader checking it by eye: no blocking, no fusion, no symmetry tricks.
 * Readings of garbled or silent passages are marked "reading:".
 *
 * Layout (this file's own choice): populations f[cell*39 + i], g[cell*39 + i];
 * multipliers lam[cell*13 + k]; cell = x + nx*(y + ny*z).
 * Mask codes: 0 fluid, 1 solid (half-way bounce-back), 2 freestream
 * (equilibrium at the far-field state), 3 outflow (zero-gradient copy along x).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q 39   /* velocities of D3Q39 (Sec. 3) */
#define NM 13  /* constraints / multipliers (Eq. 13constraints) */
#define DIM 3

enum { M_FLUID = 0, M_SOLID = 1, M_FREE = 2, M_OUT = 3 };

typedef struct {
  int32_t nx, ny, nz;
  int32_t periodic[3];
  double gamma;        /* heat-capacity ratio; C_v = 1/(gamma-1) (Sec. 2) */
  double tau;          /* BGK relaxation time, tau_f = tau_g (Pr = 1, Sec. 3) */
  int32_t kn_sensor;   /* 1: tau(eps) = tau*alpha(eps) (Eq. alpha) */
  double newton_tol;   /* stop when max |G_k| < tol (Sec. 5 step table) */
  int32_t newton_maxit;
  int32_t newton_min_upd; /* reading: at least this many updates per solve */
  double rho_inf, u_inf[3], T_inf; /* far-field state for freestream cells */
  double prandtl;      /* Prandtl number; 0 or 1: Pr = 1, plain BGK (Sec. 3) */
  int32_t root_finder; /* 0: Newton-Raphson (Sec. 3); 1: chord-Newton hybrid; 2: Newton with a
                          float direction; 3: 2 after a single-precision start (other root
                          finders: Sec. 6 outlook) */
} o39_params;

typedef struct {
  int64_t fluid_cells;
  int64_t failed_cells;
  int64_t newton_updates;  /* summed over fluid cells */
  int64_t hist[32];        /* cells by number of Newton updates (clipped) */
  int64_t eps_hist[4];     /* cells by alpha branch */
} o39_stats;

/* ---------------------------------------------------------------------- */
/* Lattice (Sec. 3): D3Q39 = Shan's E^39_{3,7}: (0,0,0), (1,0,0)_FS,
 * (+-1,+-1,+-1), (2,0,0)_FS, (2,2,0)_FS, (3,0,0)_FS.  "FS" = all sign and
 * axis permutations.  Enumerated over [-3,3]^3 in lexicographic order.      */
static int VEL[Q][DIM];
static int OPP[Q];
static double WGT[Q];
static int lattice_ready = 0;

static int shell_of(int a, int b, int c) {
  /* sorted absolute components identify the shell; -1 = not in D3Q39 */
  int v[3] = {abs(a), abs(b), abs(c)};
  for (int i = 0; i < 3; ++i)
    for (int j = i + 1; j < 3; ++j)
      if (v[j] < v[i]) { int t = v[i]; v[i] = v[j]; v[j] = t; }
  if (v[0] == 0 && v[1] == 0 && v[2] == 0) return 0;
  if (v[0] == 0 && v[1] == 0 && v[2] == 1) return 1;
  if (v[0] == 1 && v[1] == 1 && v[2] == 1) return 2;
  if (v[0] == 0 && v[1] == 0 && v[2] == 2) return 3;
  if (v[0] == 0 && v[1] == 2 && v[2] == 2) return 4;
  if (v[0] == 0 && v[1] == 0 && v[2] == 3) return 5;
  return -1;
}

/* Shan's quadrature weights for E^39_{3,7}, per shell.  The method itself is
 * quadrature-free and never uses them (Sec. 2, after Eq. constraints); they
 * are exported as lattice metadata only. */
static const double SHELL_W[6] = {1.0 / 12.0, 1.0 / 12.0, 1.0 / 27.0,
                                  2.0 / 135.0, 1.0 / 432.0, 1.0 / 1620.0};

static void build_lattice(void) {
  if (lattice_ready) return;
  int n = 0;
  for (int a = -3; a <= 3; ++a)
    for (int b = -3; b <= 3; ++b)
      for (int c = -3; c <= 3; ++c) {
        int s = shell_of(a, b, c);
        if (s < 0) continue;
        VEL[n][0] = a; VEL[n][1] = b; VEL[n][2] = c;
        WGT[n] = SHELL_W[s];
        ++n;
      }
  for (int i = 0; i < Q; ++i)
    for (int j = 0; j < Q; ++j)
      if (VEL[j][0] == -VEL[i][0] && VEL[j][1] == -VEL[i][1] && VEL[j][2] == -VEL[i][2])
        OPP[i] = j;
  lattice_ready = (n == Q);
}

int o39_lattice(int32_t *vel, double *w, int32_t *opp) {
  build_lattice();
  for (int i = 0; i < Q; ++i) {
    for (int d = 0; d < DIM; ++d) vel[3 * i + d] = VEL[i][d];
    w[i] = WGT[i];
    opp[i] = OPP[i];
  }
  return lattice_ready ? Q : -1;
}

/* ---------------------------------------------------------------------- */
/* Moment basis of Eq. (discrete-equilibrium): the 13 monomials whose
 * multipliers appear in the exponent,
 *   phi = [1, xi_x, xi_y, xi_z, xi_x^2, xi_y^2, xi_z^2, xi_x xi_y, xi_x xi_z,
 *          xi_y xi_z, xi_x |xi|^2, xi_y |xi|^2, xi_z |xi|^2].
 * The off-diagonal entries of the symmetric tensor lambda_2 appear twice in
 * lambda_2:xi xi; here their sum is one multiplier (same function space). */
void o39_basis(const int32_t *xi, double *phi) {
  double x = xi[0], y = xi[1], z = xi[2];
  double s = x * x + y * y + z * z;
  phi[0] = 1.0;
  phi[1] = x; phi[2] = y; phi[3] = z;
  phi[4] = x * x; phi[5] = y * y; phi[6] = z * z;
  phi[7] = x * y; phi[8] = x * z; phi[9] = y * z;
  phi[10] = x * s; phi[11] = y * s; phi[12] = z * s;
}

static void basis_i(int i, double *phi) {
  int32_t xi[3] = {VEL[i][0], VEL[i][1], VEL[i][2]};
  o39_basis(xi, phi);
}

/* Targets, Eq. (13constraints), divided by rho:
 *   M0 = 1; M1_a = u_a; M2_ab = u_a u_b + T delta_ab;
 *   M3_a = sum_b M3_abb = u_a (u^2 + (D+2) T).
 * reading: the printed right-hand side "(2 rho E^tr + 2 rho T) u_a" with
 * "E^tr = D T + rho u^2" is dimensionally garbled; the contracted third
 * moment of the Maxwell-Boltzmann distribution (Eq. EqMomentsTensor,
 * contracted over beta = gamma) is rho u_a (u^2 + (D+2) T), which equals the
 * printed form for rho E^tr = rho u^2 / 2 + D rho T / 2. */
void o39_targets(const double *u, double T, double *m) {
  double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  m[0] = 1.0;
  m[1] = u[0]; m[2] = u[1]; m[3] = u[2];
  m[4] = u[0] * u[0] + T; m[5] = u[1] * u[1] + T; m[6] = u[2] * u[2] + T;
  m[7] = u[0] * u[1]; m[8] = u[0] * u[2]; m[9] = u[1] * u[2];
  m[10] = u[0] * (u2 + (DIM + 2) * T);
  m[11] = u[1] * (u2 + (DIM + 2) * T);
  m[12] = u[2] * (u2 + (DIM + 2) * T);
}

/* Normalised exponential equilibrium, Eq. (discrete-equilibrium) / rho:
 *   F_i = exp(sum_k lam_k phi_k(xi_i)),  f_i^eq = rho F_i. */
void o39_feq_norm(const double *lam, double *F) {
  build_lattice();
  for (int i = 0; i < Q; ++i) {
    double phi[NM];
    basis_i(i, phi);
    double e = 0.0;
    for (int k = 0; k < NM; ++k) e += lam[k] * phi[k];
    F[i] = exp(e);
  }
}

/* Constraint residual, Eq. (constraints): G_k = sum_i F_i phi_k(xi_i) - m_k. */
static void residual_from_F(const double *F, const double *m, double *G) {
  for (int k = 0; k < NM; ++k) {
    double s = 0.0;
    for (int i = 0; i < Q; ++i) {
      double phi[NM];
      basis_i(i, phi);
      s += F[i] * phi[k];
    }
    G[k] = s - m[k];
  }
}

void o39_residual(const double *lam, const double *m, double *G) {
  double F[Q];
  o39_feq_norm(lam, F);
  residual_from_F(F, m, G);
}

/* Jacobian of G w.r.t. lambda (Sec. 5 step table): J_kl = sum_i F_i phi_k phi_l. */
static void jacobian_from_F(const double *F, double *J) {
  for (int k = 0; k < NM; ++k)
    for (int l = 0; l < NM; ++l) {
      double s = 0.0;
      for (int i = 0; i < Q; ++i) {
        double phi[NM];
        basis_i(i, phi);
        s += F[i] * phi[k] * phi[l];
      }
      J[k * NM + l] = s;
    }
}

void o39_jacobian(const double *lam, double *J) {
  double F[Q];
  o39_feq_norm(lam, F);
  jacobian_from_F(F, J);
}

/* Inverse of the n x n matrix Jin (n <= NM) by textbook Gauss-Jordan
 * elimination with partial pivoting.  Returns 0, or -1 if singular. */
static int invert_n(const double *Jin, double *Jinv, int n) {
  double a[NM][2 * NM];
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) {
      a[r][c] = Jin[r * n + c];
      a[r][n + c] = (r == c) ? 1.0 : 0.0;
    }
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(a[r][c]) > fabs(a[p][c])) p = r;
    if (!(fabs(a[p][c]) > 0.0)) return -1;
    if (p != c)
      for (int k = 0; k < 2 * n; ++k) { double t = a[c][k]; a[c][k] = a[p][k]; a[p][k] = t; }
    double piv = a[c][c];
    for (int k = 0; k < 2 * n; ++k) a[c][k] /= piv;
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double fct = a[r][c];
      if (fct == 0.0) continue;
      for (int k = 0; k < 2 * n; ++k) a[r][k] -= fct * a[c][k];
    }
  }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) Jinv[r * n + c] = a[r][n + c];
  return 0;
}

/* "Compute inverse of J" (Sec. 5 step table). */
int o39_invert(const double *Jin, double *Jinv) { return invert_n(Jin, Jinv, NM); }

static double maxabs(const double *v) {
  double r = 0.0;
  for (int k = 0; k < NM; ++k) {
    double a = fabs(v[k]);
    if (!(a <= r)) r = a; /* NaN propagates */
  }
  return r;
}

static double sumsq(const double *v) {
  double s = 0.0;
  for (int k = 0; k < NM; ++k) s += v[k] * v[k];
  return s;
}

/* Gaussian starting point for a cold start.
 * reading (the paper only says lambda is inherited from the previous step):
 * lam_1 = u/T, diagonal lam_2 = -1/(2T), everything else 0, and lam_0
 * normalises sum_i F_i = 1 -- the discrete Maxwellian exp(-(xi-u)^2/(2T)). */
void o39_gaussian_guess(const double *u, double T, double *lam) {
  build_lattice();
  for (int k = 0; k < NM; ++k) lam[k] = 0.0;
  lam[1] = u[0] / T; lam[2] = u[1] / T; lam[3] = u[2] / T;
  lam[4] = lam[5] = lam[6] = -0.5 / T;
  double F[Q];
  o39_feq_norm(lam, F);
  double s = 0.0;
  for (int i = 0; i < Q; ++i) s += F[i];
  lam[0] = -log(s);
}

#define LS_MAX 30
#define N5 5               /* constraints of the fallback equilibrium */
#define FALLBACK_MAXIT 50  /* Newton updates of the fallback from its Gaussian start */
#define FALLBACK_TOL 1e-12
#define RETRY_PERIOD 8     /* a cell on the fallback retries the full solve on steps t = 0 mod this */

/* Newton-Raphson for the 13 multipliers (Sec. 3 and the Sec. 5 step table):
 * repeat { F = exp(Phi lam); G = Phi^T F - m; J = Phi^T diag(F) Phi;
 *          lam <- lam - J^{-1} G } until max|G| < tol.
 * reading (stopping and damping are not specified beyond "norm below 1e-12"):
 *  - at least `min_upd` updates are taken (default 0: a warm start whose
 *    residual is already at round-off takes none, as the paper reports for
 *    wide areas of its airfoil flow, Sec. 4);
 *  - a solve that lands between tol/100 and tol (above the round-off floor of
 *    the residual) takes one more full "polishing" step from there; with
 *    quadratic convergence that step ends at round-off, so the collision
 *    conserves mass, momentum and energy to round-off;
 *  - while not converged, the step is halved until ||G||_2 decreases
 *    (backtracking), which keeps a cold start from overflowing;
 *  - more than `maxit` updates, or no decrease within LS_MAX halvings, is a
 *    failure (return 1; lam keeps its last accepted value).
 * On return F holds exp(Phi lam) at the returned lam. */
int o39_newton(const double *m, double *lam, double tol, int maxit, int min_upd,
               int *n_upd_out, double *F) {
  build_lattice();
  double G[NM];
  o39_feq_norm(lam, F);
  residual_from_F(F, m, G);
  int n_upd = 0, status = 0, polished = 0;
  for (;;) {
    double r = maxabs(G);
    if (n_upd >= min_upd && r < tol && (r < 1e-2 * tol || polished)) break;
    if (n_upd >= maxit) { status = 1; break; }
    double J[NM * NM], Ji[NM * NM], d[NM];
    jacobian_from_F(F, J);
    if (o39_invert(J, Ji) != 0) { status = 1; break; }
    for (int k = 0; k < NM; ++k) {
      double s = 0.0;
      for (int l = 0; l < NM; ++l) s += Ji[k * NM + l] * G[l];
      d[k] = s;
    }
    double lt[NM], Ft[Q], Gt[NM];
    polished = (r < tol);
    if (polished) { /* polishing step: always full */
      for (int k = 0; k < NM; ++k) lt[k] = lam[k] - d[k];
      o39_feq_norm(lt, Ft);
      residual_from_F(Ft, m, Gt);
    } else {
      double s0 = sumsq(G), t = 1.0;
      int ok = 0;
      for (int ls = 0; ls <= LS_MAX; ++ls) {
        for (int k = 0; k < NM; ++k) lt[k] = lam[k] - t * d[k];
        o39_feq_norm(lt, Ft);
        residual_from_F(Ft, m, Gt);
        if (sumsq(Gt) < s0) { ok = 1; break; }
        t *= 0.5;
      }
      if (!ok) { status = 1; break; }
    }
    memcpy(lam, lt, sizeof lt);
    memcpy(F, Ft, sizeof Ft);
    memcpy(G, Gt, sizeof Gt);
    ++n_upd;
  }
  if (n_upd_out) *n_upd_out = n_upd;
  return status;
}

/* Chord-Newton hybrid for the same 13 equations (the paper's outlook, Sec. 6,
 * names other root finders; this one is the oracle's reading of a standard
 * variant).  Same stopping rule, polishing step, budget and failure rule as
 * o39_newton; the direction J^{-1} G reuses the last Jacobian formed in this
 * solve (a chord step) as long as the previous accepted step reduced max|G|
 * by at least the factor CHORD_RHO, and otherwise forms J at the current
 * point (a Newton step).  A chord step that does not reduce ||G||_2 is not
 * halved: J is formed at the current point instead and the update is retried
 * as a Newton step.  Each Jacobian formed is counted in *n_jac_out.
 * Near the root a chord step contracts the error by the relative change of J
 * since it was formed, so after a Newton step of quadratic convergence the
 * next steps can skip forming and inverting J. */
#define CHORD_RHO 1e-3

int o39_newton_hybrid(const double *m, double *lam, double tol, int maxit, int min_upd,
                      int *n_upd_out, int *n_jac_out, double *F) {
  build_lattice();
  double G[NM], Ji[NM * NM];
  o39_feq_norm(lam, F);
  residual_from_F(F, m, G);
  int n_upd = 0, n_jac = 0, status = 0, polished = 0, have_J = 0;
  double r_prev = 0.0;  /* max|G| before the last accepted step; 0: none yet */
  for (;;) {
    double r = maxabs(G);
    if (n_upd >= min_upd && r < tol && (r < 1e-2 * tol || polished)) break;
    if (n_upd >= maxit) { status = 1; break; }
    const int chord = have_J && r_prev > 0.0 && r <= CHORD_RHO * r_prev;
    if (!chord) {
      double J[NM * NM];
      jacobian_from_F(F, J);
      ++n_jac;
      if (o39_invert(J, Ji) != 0) { status = 1; break; }
      have_J = 1;
    }
    double d[NM];
    for (int k = 0; k < NM; ++k) {
      double s = 0.0;
      for (int l = 0; l < NM; ++l) s += Ji[k * NM + l] * G[l];
      d[k] = s;
    }
    double lt[NM], Ft[Q], Gt[NM];
    polished = (r < tol);
    if (polished) { /* polishing step: always full */
      for (int k = 0; k < NM; ++k) lt[k] = lam[k] - d[k];
      o39_feq_norm(lt, Ft);
      residual_from_F(Ft, m, Gt);
    } else {
      double s0 = sumsq(G), t = 1.0;
      int ok = 0;
      for (int ls = 0; ls <= LS_MAX; ++ls) {
        for (int k = 0; k < NM; ++k) lt[k] = lam[k] - t * d[k];
        o39_feq_norm(lt, Ft);
        residual_from_F(Ft, m, Gt);
        if (sumsq(Gt) < s0) { ok = 1; break; }
        if (chord) break; /* a chord step is not halved */
        t *= 0.5;
      }
      if (!ok && chord) { /* retry from here with J formed at this point */
        have_J = 0;
        r_prev = 0.0;
        polished = 0;
        continue;
      }
      if (!ok) { status = 1; break; }
    }
    r_prev = r;
    memcpy(lam, lt, sizeof lt);
    memcpy(F, Ft, sizeof Ft);
    memcpy(G, Gt, sizeof Gt);
    ++n_upd;
  }
  if (n_upd_out) *n_upd_out = n_upd;
  if (n_jac_out) *n_jac_out = n_jac;
  return status;
}

/* Inverse of the n x n matrix Jin (n <= NM) in single precision: textbook
 * Gauss-Jordan elimination with partial pivoting, every operation in float.
 * Returns 0, or -1 if singular. */
static int invert_float(const float *Jin, float *Jinv, int n) {
  float a[NM][2 * NM];
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) {
      a[r][c] = Jin[r * n + c];
      a[r][n + c] = (r == c) ? 1.0f : 0.0f;
    }
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (fabsf(a[r][c]) > fabsf(a[p][c])) p = r;
    if (!(fabsf(a[p][c]) > 0.0f)) return -1;
    if (p != c)
      for (int k = 0; k < 2 * n; ++k) { float t = a[c][k]; a[c][k] = a[p][k]; a[p][k] = t; }
    float piv = a[c][c];
    for (int k = 0; k < 2 * n; ++k) a[c][k] /= piv;
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      float fct = a[r][c];
      if (fct == 0.0f) continue;
      for (int k = 0; k < 2 * n; ++k) a[r][k] -= fct * a[c][k];
    }
  }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) Jinv[r * n + c] = a[r][n + c];
  return 0;
}

/* Newton with a single-precision direction (a third root finder; the
 * paper's outlook names other root finders): the same stopping rule,
 * polishing step, budget, line search and failure rule as o39_newton, with
 * the residual G and the update of lam in double precision, but the
 * direction d = J^{-1} G formed in float: F and G rounded to float, J summed
 * and inverted in float.  An inexact Newton iteration (iterative refinement):
 * each step contracts the residual by about cond(J) times the float
 * precision instead of squaring it, and it converges to the same equilibrium,
 * because the residual that decides convergence is the double-precision one. */
int o39_newton_fp32dir(const double *m, double *lam, double tol, int maxit, int min_upd,
                       int *n_upd_out, double *F) {
  build_lattice();
  double G[NM];
  o39_feq_norm(lam, F);
  residual_from_F(F, m, G);
  int n_upd = 0, status = 0, polished = 0;
  for (;;) {
    double r = maxabs(G);
    if (n_upd >= min_upd && r < tol && (r < 1e-2 * tol || polished)) break;
    if (n_upd >= maxit) { status = 1; break; }
    float J[NM * NM], Ji[NM * NM], Gf[NM];
    for (int k = 0; k < NM; ++k)
      for (int l = 0; l < NM; ++l) {
        float s = 0.0f;
        for (int i = 0; i < Q; ++i) {
          double phi[NM];
          basis_i(i, phi);
          s += (float)F[i] * (float)phi[k] * (float)phi[l];
        }
        J[k * NM + l] = s;
      }
    if (invert_float(J, Ji, NM) != 0) { status = 1; break; }
    for (int k = 0; k < NM; ++k) Gf[k] = (float)G[k];
    double d[NM];
    for (int k = 0; k < NM; ++k) {
      float s = 0.0f;
      for (int l = 0; l < NM; ++l) s += Ji[k * NM + l] * Gf[l];
      d[k] = s;
    }
    double lt[NM], Ft[Q], Gt[NM];
    polished = (r < tol);
    if (polished) {
      for (int k = 0; k < NM; ++k) lt[k] = lam[k] - d[k];
      o39_feq_norm(lt, Ft);
      residual_from_F(Ft, m, Gt);
    } else {
      double s0 = sumsq(G), t = 1.0;
      int ok = 0;
      for (int ls = 0; ls <= LS_MAX; ++ls) {
        for (int k = 0; k < NM; ++k) lt[k] = lam[k] - t * d[k];
        o39_feq_norm(lt, Ft);
        residual_from_F(Ft, m, Gt);
        if (sumsq(Gt) < s0) { ok = 1; break; }
        t *= 0.5;
      }
      if (!ok) { status = 1; break; }
    }
    memcpy(lam, lt, sizeof lt);
    memcpy(F, Ft, sizeof Ft);
    memcpy(G, Gt, sizeof Gt);
    ++n_upd;
  }
  if (n_upd_out) *n_upd_out = n_upd;
  return status;
}

/* Newton started in single precision (a fourth root finder; the outlook,
 * Sec. 6, names other root finders).  reading: from a warm start the first
 * Newton steps only need the residual to a few digits, which float
 * arithmetic gives; the last digits need double precision.  So:
 *  1. from F0 = exp(Phi lam) (double, rounded to float), Newton steps in float
 *     on the change delta of the multipliers: F_i = F0_i expf(phi(xi_i).delta),
 *     G = sum_i F_i phi(xi_i) - m, J = sum_i F_i phi phi^T, delta <- delta - J^{-1} G,
 *     every operation in float, while max|G| >= START32_THETA and at most
 *     START32_MAXIT times; a step is kept only if it lowers max|G| (otherwise
 *     this phase ends there, with the last kept delta);
 *  2. lam <- lam + delta in double, then o39_newton_fp32dir from there, whose
 *     double-precision residual decides convergence as for every root finder.
 * A solve with no budget (maxit = 0: a cell on the fallback off a retry step)
 * takes no float step either.  *n32_out: the float steps kept. */
#define START32_THETA 1e-4f
#define START32_MAXIT 4

static void eval_float(const float *F0, const float *delta, const float *mf, float *F,
                       float *G) {
  for (int i = 0; i < Q; ++i) {
    double phi[NM];
    basis_i(i, phi);
    float e = 0.0f;
    for (int k = 0; k < NM; ++k) e += delta[k] * (float)phi[k];
    F[i] = F0[i] * expf(e);
  }
  for (int k = 0; k < NM; ++k) {
    float s = 0.0f;
    for (int i = 0; i < Q; ++i) {
      double phi[NM];
      basis_i(i, phi);
      s += F[i] * (float)phi[k];
    }
    G[k] = s - mf[k];
  }
}

static float maxabs_float(const float *v) {
  float r = 0.0f;
  for (int k = 0; k < NM; ++k) {
    float a = fabsf(v[k]);
    if (!(a <= r)) r = a;
  }
  return r;
}

int o39_newton_fp32start(const double *m, double *lam, double tol, int maxit, int min_upd,
                         int *n_upd_out, int *n32_out, double *F) {
  build_lattice();
  int n32 = 0;
  if (maxit > 0) {
    double F0d[Q];
    float F0[Q], mf[NM], delta[NM], Fc[Q], G[NM];
    o39_feq_norm(lam, F0d);
    for (int i = 0; i < Q; ++i) F0[i] = (float)F0d[i];
    for (int k = 0; k < NM; ++k) { mf[k] = (float)m[k]; delta[k] = 0.0f; }
    eval_float(F0, delta, mf, Fc, G);
    float r = maxabs_float(G);
    while (n32 < START32_MAXIT && r >= START32_THETA) {
      float J[NM * NM], Ji[NM * NM], dt[NM], Ft[Q], Gt[NM];
      for (int k = 0; k < NM; ++k)
        for (int l = 0; l < NM; ++l) {
          float s = 0.0f;
          for (int i = 0; i < Q; ++i) {
            double phi[NM];
            basis_i(i, phi);
            s += Fc[i] * (float)phi[k] * (float)phi[l];
          }
          J[k * NM + l] = s;
        }
      if (invert_float(J, Ji, NM) != 0) break;
      for (int k = 0; k < NM; ++k) {
        float s = 0.0f;
        for (int l = 0; l < NM; ++l) s += Ji[k * NM + l] * G[l];
        dt[k] = delta[k] - s;
      }
      eval_float(F0, dt, mf, Ft, Gt);
      float rt = maxabs_float(Gt);
      if (!(rt < r)) break;
      memcpy(delta, dt, sizeof dt);
      memcpy(Fc, Ft, sizeof Ft);
      memcpy(G, Gt, sizeof Gt);
      r = rt;
      ++n32;
    }
    for (int k = 0; k < NM; ++k) lam[k] += (double)delta[k];
  }
  if (n32_out) *n32_out = n32;
  return o39_newton_fp32dir(m, lam, tol, maxit, min_upd, n_upd_out, F);
}

/* The root finder the run parameters select. */
static int solve13(const o39_params *p, const double *m, double *lam, int maxit, int *n_upd,
                   double *F) {
  if (p->root_finder == 1)
    return o39_newton_hybrid(m, lam, p->newton_tol, maxit, p->newton_min_upd, n_upd, NULL, F);
  if (p->root_finder == 2)
    return o39_newton_fp32dir(m, lam, p->newton_tol, maxit, p->newton_min_upd, n_upd, F);
  if (p->root_finder == 3)
    return o39_newton_fp32start(m, lam, p->newton_tol, maxit, p->newton_min_upd, n_upd, NULL, F);
  return o39_newton(m, lam, p->newton_tol, maxit, p->newton_min_upd, n_upd, F);
}

/* ---------------------------------------------------------------------- */
/* Fallback where the 13-moment equilibrium does not exist.
 * reading (the paper does not say what a cell does when its constraint solve
 * fails): outside the moment cone of the 39 velocities no positive
 * distribution has the 13 target moments, and Newton cannot converge.  Such a
 * cell relaxes instead to the maximum-entropy equilibrium under the five
 * collision invariants phi5 = [1, xi, |xi|^2] only,
 *   F_i = exp(mu_0 + mu . xi_i + mu_4 |xi_i|^2),  sum_i F_i phi5(xi_i) = [1, u, u^2 + D T],
 * which exists far beyond that cone and conserves mass, momentum and energy
 * (with g^eq = (2 C_v - D) T f^eq as for the full equilibrium).  It is solved
 * by the same damped Newton iteration as the full system. */

static void basis5_i(int i, double *phi) {
  phi[0] = 1.0;
  phi[1] = VEL[i][0]; phi[2] = VEL[i][1]; phi[3] = VEL[i][2];
  phi[4] = VEL[i][0] * VEL[i][0] + VEL[i][1] * VEL[i][1] + VEL[i][2] * VEL[i][2];
}

void o39_targets5(const double *u, double T, double *m) {
  m[0] = 1.0;
  m[1] = u[0]; m[2] = u[1]; m[3] = u[2];
  m[4] = u[0] * u[0] + u[1] * u[1] + u[2] * u[2] + DIM * T;
}

void o39_feq5(const double *mu, double *F) {
  build_lattice();
  for (int i = 0; i < Q; ++i) {
    double phi[N5];
    basis5_i(i, phi);
    double e = 0.0;
    for (int k = 0; k < N5; ++k) e += mu[k] * phi[k];
    F[i] = exp(e);
  }
}

static void residual5(const double *F, const double *m, double *G) {
  for (int k = 0; k < N5; ++k) {
    double s = 0.0;
    for (int i = 0; i < Q; ++i) {
      double phi[N5];
      basis5_i(i, phi);
      s += F[i] * phi[k];
    }
    G[k] = s - m[k];
  }
}

static double maxabs_n(const double *v, int n) {
  double r = 0.0;
  for (int k = 0; k < n; ++k) {
    double a = fabs(v[k]);
    if (!(a <= r)) r = a;
  }
  return r;
}

static double sumsq_n(const double *v, int n) {
  double s = 0.0;
  for (int k = 0; k < n; ++k) s += v[k] * v[k];
  return s;
}

/* Gaussian start: mu = (., u/T, -1/(2T)), mu_0 normalising sum_i F_i = 1. */
void o39_gaussian_guess5(const double *u, double T, double *mu) {
  build_lattice();
  mu[0] = 0.0;
  mu[1] = u[0] / T; mu[2] = u[1] / T; mu[3] = u[2] / T;
  mu[4] = -0.5 / T;
  double F[Q];
  o39_feq5(mu, F);
  double s = 0.0;
  for (int i = 0; i < Q; ++i) s += F[i];
  mu[0] = -log(s);
}

/* Newton for the five multipliers with the same stopping rule, polishing step
 * and backtracking as o39_newton.  Returns 0 or 1 (failure). */
int o39_newton5(const double *m, double *mu, double tol, int maxit, int *n_upd_out, double *F) {
  build_lattice();
  double G[N5];
  o39_feq5(mu, F);
  residual5(F, m, G);
  int n_upd = 0, status = 0, polished = 0;
  for (;;) {
    double r = maxabs_n(G, N5);
    if (r < tol && (r < 1e-2 * tol || polished)) break;
    if (n_upd >= maxit) { status = 1; break; }
    double J[N5 * N5], Ji[N5 * N5], d[N5];
    for (int k = 0; k < N5; ++k)
      for (int l = 0; l < N5; ++l) {
        double s = 0.0;
        for (int i = 0; i < Q; ++i) {
          double phi[N5];
          basis5_i(i, phi);
          s += F[i] * phi[k] * phi[l];
        }
        J[k * N5 + l] = s;
      }
    if (invert_n(J, Ji, N5) != 0) { status = 1; break; }
    for (int k = 0; k < N5; ++k) {
      double s = 0.0;
      for (int l = 0; l < N5; ++l) s += Ji[k * N5 + l] * G[l];
      d[k] = s;
    }
    double mt[N5], Ft[Q], Gt[N5];
    polished = (r < tol);
    if (polished) {
      for (int k = 0; k < N5; ++k) mt[k] = mu[k] - d[k];
      o39_feq5(mt, Ft);
      residual5(Ft, m, Gt);
    } else {
      double s0 = sumsq_n(G, N5), t = 1.0;
      int ok = 0;
      for (int ls = 0; ls <= LS_MAX; ++ls) {
        for (int k = 0; k < N5; ++k) mt[k] = mu[k] - t * d[k];
        o39_feq5(mt, Ft);
        residual5(Ft, m, Gt);
        if (sumsq_n(Gt, N5) < s0) { ok = 1; break; }
        t *= 0.5;
      }
      if (!ok) { status = 1; break; }
    }
    memcpy(mu, mt, sizeof mt);
    memcpy(F, Ft, sizeof Ft);
    memcpy(G, Gt, sizeof Gt);
    ++n_upd;
  }
  if (n_upd_out) *n_upd_out = n_upd;
  return status;
}

/* Failure policy (reading; the paper is silent).  A cell whose full solve
 * fails takes the fallback equilibrium and keeps its five multipliers
 * embedded in the 13,
 *   lam = (mu_0, mu_x, mu_y, mu_z, mu_4, mu_4, mu_4, 0, 0, 0, 0, 0, 0),
 * for which exp(Phi lam) is the fallback equilibrium (|xi|^2 = xi_x^2 +
 * xi_y^2 + xi_z^2), and a per-cell flag "on the fallback" is set.  On the
 * next steps a flagged cell does not repeat the full solve from scratch:
 *  - on every step t that is a multiple of RETRY_PERIOD it tries the full
 *    solve again from the embedding, with the full Newton budget; a cell
 *    that has come back inside the cone converges and its flag is cleared;
 *  - on the other steps it takes no update (only the residual of the
 *    embedding is checked), and the fallback starts from the stored mu.
 * Cells outside the cone usually stay outside for many steps (the region is
 * carried by the flow), so this limits the work of a cell that cannot
 * converge to one full attempt every RETRY_PERIOD steps and a fallback solve
 * from a close start, while a cell that has re-entered the cone returns to
 * the 13-moment equilibrium within RETRY_PERIOD steps.  The retry needs the
 * full budget: from the five-multiplier embedding the full solve takes 5 to 7
 * updates even for states well inside the cone (|u| ~ 1, T ~ 0.5), so a
 * shorter budget keeps such cells on the fallback for good.  The rule depends
 * on the time step alone.  If the
 * fallback fails as well, the cell keeps the multipliers the full solve left,
 * its equilibrium is evaluated there, and its flag is cleared. */

/* The fallback for the state (u, T), from the stored mu (warm, the first five
 * entries of an embedding) or the Gaussian start (warm NULL).  On success lam
 * becomes the embedding of its multipliers and F = exp(Phi lam); otherwise
 * lam and F are left as they are.  Returns the fallback's status. */
static int fallback_into(const double *u, double T, const double *warm, double *lam, double *F) {
  double m5[N5], mu[N5], F5[Q];
  o39_targets5(u, T, m5);
  if (warm) {
    for (int k = 0; k < N5; ++k) mu[k] = warm[k];
  } else {
    o39_gaussian_guess5(u, T, mu);
  }
  if (o39_newton5(m5, mu, FALLBACK_TOL, FALLBACK_MAXIT, NULL, F5) != 0) return 1;
  for (int k = 0; k < NM; ++k) lam[k] = 0.0;
  for (int k = 0; k < 4; ++k) lam[k] = mu[k];
  lam[4] = lam[5] = lam[6] = mu[4];
  o39_feq_norm(lam, F);
  return 0;
}

/* alpha(eps), Eq. (alpha): 1 below 1e-2, 1.05 on [1e-2,1e-1), 1.35 on
 * [1e-1,1), and 1/tau from 1 upward (then tau*alpha = 1: h* = h^eq). */
double o39_alpha(double eps, double tau) {
  if (eps < 1e-2) return 1.0;
  if (eps < 1e-1) return 1.05;
  if (eps < 1.0) return 1.35;
  return 1.0 / tau;
}

static int alpha_branch(double eps) {
  if (eps < 1e-2) return 0;
  if (eps < 1e-1) return 1;
  if (eps < 1.0) return 2;
  return 3;
}

/* Macroscopic variables of one cell (Sec. 3, first collision step):
 * rho = sum f, rho u = sum f xi, and T from the total energy
 *   sum f |xi|^2 + sum g = rho u^2 + 2 C_v rho T    (E = u^2/2 + C_v T, Sec. 2).
 * reading: T is taken from the total energy of both populations, which is
 * what makes g^eq = (2C_v - D) T f^eq conserve energy. */
void o39_cell_macros(const o39_params *p, const double *f, const double *g,
                     double *rho_out, double *u_out, double *T_out) {
  build_lattice();
  double cv = 1.0 / (p->gamma - 1.0);
  double rho = 0.0, j[3] = {0, 0, 0}, e2 = 0.0;
  for (int i = 0; i < Q; ++i) {
    rho += f[i];
    for (int d = 0; d < DIM; ++d) j[d] += f[i] * VEL[i][d];
    double c2 = VEL[i][0] * VEL[i][0] + VEL[i][1] * VEL[i][1] + VEL[i][2] * VEL[i][2];
    e2 += f[i] * c2 + g[i];
  }
  double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
  double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  *rho_out = rho;
  for (int d = 0; d < DIM; ++d) u_out[d] = u[d];
  *T_out = (e2 - rho * u2) / (2.0 * cv * rho);
}

/* Prandtl-number adjustment (Sec. 3 names it -- a quasi-equilibrium, or a
 * temperature-scaled collision -- and leaves it out, so that Pr = 1; the
 * formulas here are this oracle's reading, written from the mathematics).
 *
 * Quasi-equilibrium collision with two relaxation times: each population
 * relaxes towards a quasi-equilibrium h* with 1/tau and h* towards h^eq with
 * 1/tau2,
 *   h' = h - (h - h^eq)/tau + (1/tau - 1/tau2) (h* - h^eq),   h = f, g.
 * The quasi-equilibrium keeps f* = f^eq and differs from the equilibrium only
 * in the heat flux, which it takes from the current populations: with the
 * peculiar velocity c_i = xi_i - u, the heat flux is
 *   q = (1/2) sum_i c_i (|c_i|^2 f_i + g_i),
 * which is zero at the 13-moment equilibrium (its contracted third moment is
 * the Maxwellian's, Eq. 13constraints, and sum_i c_i g^eq_i = 0), and
 *   g*_i - g^eq_i = dg_i = g^eq_i (c_i . b),  b = 2 q / ((2 C_v - D) rho T^2),
 * so that (1/2) sum_i c_i dg_i = q (because sum_i f^eq_i c_i c_i = rho T I at
 * the equilibrium), while sum_i dg_i = 0 (no energy moves) and f is not
 * touched (mass and momentum untouched).  After one collision the heat flux is
 * (1 - 1/tau2) q and the stress relaxes with 1/tau as before, so to first
 * order in the Chapman-Enskog expansion the viscosity goes with (tau - 1/2)
 * and the heat conductivity with (tau2 - 1/2): Pr = (tau - 1/2)/(tau2 - 1/2).
 * reading: tau2 follows the relaxation time actually used, tau_eff = tau
 * alpha(eps), as tau2 = 1/2 + (tau_eff - 1/2)/Pr, so the sensor of Eq. (alpha)
 * keeps the Prandtl number.  Needs 2 C_v - D > 0 (g^eq nonzero). */
static double heat_flux_tau(const o39_params *p, double tau_eff) {
  if (p->prandtl == 0.0 || p->prandtl == 1.0) return tau_eff;
  return 0.5 + (tau_eff - 0.5) / p->prandtl;
}

static void prandtl_correction(const o39_params *p, const double *f, const double *g,
                               const double *geq, double rho, const double *u, double T,
                               double *dg) {
  for (int i = 0; i < Q; ++i) dg[i] = 0.0;
  if (p->prandtl == 0.0 || p->prandtl == 1.0) return;
  double cv = 1.0 / (p->gamma - 1.0);
  double q[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < Q; ++i) {
    double c[3] = {VEL[i][0] - u[0], VEL[i][1] - u[1], VEL[i][2] - u[2]};
    double c2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
    for (int a = 0; a < DIM; ++a) q[a] += 0.5 * c[a] * (c2 * f[i] + g[i]);
  }
  double b[3];
  for (int a = 0; a < DIM; ++a) b[a] = 2.0 * q[a] / ((2.0 * cv - DIM) * rho * T * T);
  for (int i = 0; i < Q; ++i) {
    double cb = 0.0;
    for (int a = 0; a < DIM; ++a) cb += (VEL[i][a] - u[a]) * b[a];
    dg[i] = geq[i] * cb;
  }
}

/* One BGK collision of one fluid cell (Sec. 3 and Eq. DeltaAvg / alpha):
 * macros -> MB targets -> Newton (warm start lam) -> f^eq, g^eq = (2C_v-D) T f^eq
 * -> eps, alpha -> h* = h - (h - h^eq)/(tau alpha) for h = f and h = g
 * (with the Prandtl-number adjustment above when p->prandtl is not 1).
 * t: the time step being taken; on_fb: the cell's "on the fallback" flag (in
 * and out), which with t decides the solve's budget (failure policy above).
 * reading: eps uses f only and the same alpha relaxes f and g (Pr = 1).
 * In place on f, g, lam, on_fb.  Returns the Newton status. */
int o39_collide_cell(const o39_params *p, double *f, double *g, double *lam, uint8_t *on_fb,
                     int64_t t, int *n_upd, double *eps_out, double *alpha_out) {
  build_lattice();
  double cv = 1.0 / (p->gamma - 1.0);
  double rho, u[3], T;
  o39_cell_macros(p, f, g, &rho, u, &T);
  double m[NM], F[Q];
  o39_targets(u, T, m);
  double lam_in[NM];
  memcpy(lam_in, lam, sizeof lam_in);
  const int flagged = *on_fb != 0;
  int maxit = p->newton_maxit;
  if (flagged) maxit = (t % RETRY_PERIOD == 0) ? p->newton_maxit : 0;
  int st = solve13(p, m, lam, maxit, n_upd, F);
  if (st) {  /* counted as a failure: the cell takes the fallback this step */
    if (fallback_into(u, T, flagged ? lam_in : NULL, lam, F) == 0) {
      *on_fb = 1;
    } else {
      o39_feq_norm(lam, F);
      *on_fb = 0;
    }
  } else {
    *on_fb = 0;
  }
  double feq[Q], geq[Q];
  for (int i = 0; i < Q; ++i) {
    feq[i] = rho * F[i];
    geq[i] = (2.0 * cv - DIM) * T * feq[i];
  }
  double eps = 0.0;
  for (int i = 0; i < Q; ++i) eps += fabs(f[i] - feq[i]) / feq[i];
  eps /= Q;
  double alpha = p->kn_sensor ? o39_alpha(eps, p->tau) : 1.0;
  double tau_eff = p->tau * alpha;
  double dg[Q];
  prandtl_correction(p, f, g, geq, rho, u, T, dg);
  double tau2 = heat_flux_tau(p, tau_eff);
  for (int i = 0; i < Q; ++i) {
    f[i] = f[i] - (f[i] - feq[i]) / tau_eff;
    g[i] = g[i] - (g[i] - geq[i]) / tau_eff + (1.0 / tau_eff - 1.0 / tau2) * dg[i];
  }
  if (eps_out) *eps_out = eps;
  if (alpha_out) *alpha_out = alpha;
  return st;
}

/* Equilibrium populations and multipliers of a state (rho, u, T) from the
 * Gaussian cold start (used for initial conditions and far-field cells).
 * on_fb (may be NULL): set to 1 where the fallback equilibrium was taken. */
int o39_equilibrium(const o39_params *p, double rho, const double *u, double T,
                    double *feq, double *geq, double *lam, int maxit, uint8_t *on_fb) {
  build_lattice();
  double cv = 1.0 / (p->gamma - 1.0);
  double m[NM], F[Q];
  o39_targets(u, T, m);
  o39_gaussian_guess(u, T, lam);
  int nu = 0;
  int st = o39_newton(m, lam, p->newton_tol, maxit, p->newton_min_upd, &nu, F);
  int fb = 0;
  if (st) fb = fallback_into(u, T, NULL, lam, F) == 0;
  if (on_fb) *on_fb = (uint8_t)fb;
  for (int i = 0; i < Q; ++i) {
    feq[i] = rho * F[i];
    geq[i] = (2.0 * cv - DIM) * T * feq[i];
  }
  return st;
}

/* ---------------------------------------------------------------------- */
/* Lattice-level operations. */

static int64_t cell_index(const o39_params *p, int x, int y, int z) {
  return (int64_t)x + (int64_t)p->nx * ((int64_t)y + (int64_t)p->ny * z);
}

static int wrap(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

/* Initial condition: every fluid cell at its local equilibrium f^eq(rho,u,T),
 * g^eq, with lam from a cold-start Newton; other cells hold zeros.
 * u is given as three planes u[d*N + cell].  on_fb: per-cell "on the
 * fallback" flags (out).  Returns the failed-cell count. */
int64_t o39_init(const o39_params *p, const uint8_t *mask, const double *rho,
                 const double *u, const double *T, double *f, double *g,
                 double *lam, uint8_t *on_fb, int maxit) {
  build_lattice();
  int64_t N = (int64_t)p->nx * p->ny * p->nz;
  int64_t failed = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : failed)
  for (int64_t c = 0; c < N; ++c) {
    on_fb[c] = 0;
    if (mask[c] != M_FLUID) {
      for (int i = 0; i < Q; ++i) { f[c * Q + i] = 0.0; g[c * Q + i] = 0.0; }
      for (int k = 0; k < NM; ++k) lam[c * NM + k] = 0.0;
      continue;
    }
    double uc[3] = {u[c], u[N + c], u[2 * N + c]};
    failed += o39_equilibrium(p, rho[c], uc, T[c], f + c * Q, g + c * Q, lam + c * NM, maxit,
                              on_fb + c);
  }
  return failed;
}

/* Post-collision value of a non-fluid source cell s in direction i.
 * reading (the paper gives the boundary kinds but not their reach on a
 * lattice with shifts up to 3): freestream cells hold h^eq at the far-field
 * state every step; an outflow cell copies the post-collision populations of
 * the cell reached by clamping its x into [3, nx-4] (zero gradient along x,
 * "first-order Neumann"). */
static double ghost_post(const o39_params *p, const uint8_t *mask, const double *post,
                         const double *heq_inf, int x, int y, int z, int i) {
  int64_t s = cell_index(p, x, y, z);
  if (mask[s] == M_FREE) return heq_inf[i];
  /* outflow */
  int xc = x < 3 ? 3 : (x > p->nx - 4 ? p->nx - 4 : x);
  int64_t c = cell_index(p, xc, y, z);
  if (mask[c] == M_FREE) return heq_inf[i];
  return post[c * Q + i];
}

/* Streaming, Eq. after Sec. 3: h_i(x + xi_i, t+1) = h*_i(x, t), written as a
 * pull: h_i(x, t+1) = h*_i(x - xi_i), with periodic wrap of the index; if
 * the source x - xi_i is solid, half-way bounce-back returns the population
 * that left x towards it: h_i(x, t+1) = h*_opp(i)(x).
 * reading (destination rule): only the end point of a link is tested; cells
 * the link passes over are not.  Only fluid cells are written. */
void o39_stream(const o39_params *p, const uint8_t *mask, const double *fpost,
                const double *gpost, const double *feq_inf, const double *geq_inf,
                double *fout, double *gout) {
  build_lattice();
  int nx = p->nx, ny = p->ny, nz = p->nz;
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        int64_t c = cell_index(p, x, y, z);
        if (mask[c] != M_FLUID) continue;
        for (int i = 0; i < Q; ++i) {
          int sx = wrap(x - VEL[i][0], nx), sy = wrap(y - VEL[i][1], ny),
              sz = wrap(z - VEL[i][2], nz);
          int64_t s = cell_index(p, sx, sy, sz);
          if (mask[s] == M_SOLID) {
            fout[c * Q + i] = fpost[c * Q + OPP[i]];
            gout[c * Q + i] = gpost[c * Q + OPP[i]];
          } else if (mask[s] == M_FLUID) {
            fout[c * Q + i] = fpost[s * Q + i];
            gout[c * Q + i] = gpost[s * Q + i];
          } else {
            fout[c * Q + i] = ghost_post(p, mask, fpost, feq_inf, sx, sy, sz, i);
            gout[c * Q + i] = ghost_post(p, mask, gpost, geq_inf, sx, sy, sz, i);
          }
        }
      }
}

/* nsteps full time steps from time t0: collide every fluid cell, then stream
 * (pull) from the post-collision array back into f, g.  on_fb: per-cell
 * "on the fallback" flags (in and out).  Returns failed Newton solves. */
int64_t o39_step(const o39_params *p, const uint8_t *mask, double *f, double *g,
                 double *lam, uint8_t *on_fb, int64_t t0, int nsteps, o39_stats *st) {
  build_lattice();
  int64_t N = (int64_t)p->nx * p->ny * p->nz;
  double *fp = (double *)malloc(sizeof(double) * N * Q);
  double *gp = (double *)malloc(sizeof(double) * N * Q);
  double feq_inf[Q], geq_inf[Q], lam_inf[NM];
  o39_equilibrium(p, p->rho_inf, p->u_inf, p->T_inf, feq_inf, geq_inf, lam_inf, 200, NULL);
  int64_t failed_total = 0;
  for (int t = 0; t < nsteps; ++t) {
    int64_t failed = 0, upd = 0, fluid = 0;
    int64_t hist[32] = {0}, ehist[4] = {0};
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : failed, upd, fluid)
    for (int64_t c = 0; c < N; ++c) {
      for (int i = 0; i < Q; ++i) { fp[c * Q + i] = f[c * Q + i]; gp[c * Q + i] = g[c * Q + i]; }
      if (mask[c] != M_FLUID) continue;
      int nu = 0;
      double eps, alpha;
      failed += o39_collide_cell(p, fp + c * Q, gp + c * Q, lam + c * NM, on_fb + c, t0 + t,
                                 &nu, &eps, &alpha);
      upd += nu;
      fluid += 1;
      int b = nu < 31 ? nu : 31;
      int eb = alpha_branch(eps);
#pragma omp atomic
      hist[b] += 1;
#pragma omp atomic
      ehist[eb] += 1;
    }
    o39_stream(p, mask, fp, gp, feq_inf, geq_inf, f, g);
    failed_total += failed;
    if (st) {
      st->fluid_cells = fluid;
      st->failed_cells += failed;
      st->newton_updates += upd;
      for (int k = 0; k < 32; ++k) st->hist[k] += hist[k];
      for (int k = 0; k < 4; ++k) st->eps_hist[k] += ehist[k];
    }
  }
  free(fp);
  free(gp);
  return failed_total;
}

/* Macroscopic fields of the pre-collision state: rho, u (3 planes), T and
 * p = rho T (ideal gas in lattice units).  Non-fluid cells read as 0. */
void o39_macros(const o39_params *p, const uint8_t *mask, const double *f,
                const double *g, double *rho, double *u, double *T, double *pr) {
  build_lattice();
  int64_t N = (int64_t)p->nx * p->ny * p->nz;
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < N; ++c) {
    if (mask[c] != M_FLUID) {
      rho[c] = 0; u[c] = 0; u[N + c] = 0; u[2 * N + c] = 0; T[c] = 0; pr[c] = 0;
      continue;
    }
    double r, uc[3], Tc;
    o39_cell_macros(p, f + c * Q, g + c * Q, &r, uc, &Tc);
    rho[c] = r; u[c] = uc[0]; u[N + c] = uc[1]; u[2 * N + c] = uc[2];
    T[c] = Tc; pr[c] = r * Tc;
  }
}

/* Lattice sums of mass, momentum and total energy (rho E = (sum f|xi|^2 + sum g)/2)
 * over fluid cells, for conservation checks. */
void o39_conserved(const o39_params *p, const uint8_t *mask, const double *f,
                   const double *g, double *out5) {
  build_lattice();
  int64_t N = (int64_t)p->nx * p->ny * p->nz;
  double s[5] = {0, 0, 0, 0, 0};
  for (int64_t c = 0; c < N; ++c) {
    if (mask[c] != M_FLUID) continue;
    for (int i = 0; i < Q; ++i) {
      double fi = f[c * Q + i];
      double c2 = VEL[i][0] * VEL[i][0] + VEL[i][1] * VEL[i][1] + VEL[i][2] * VEL[i][2];
      s[0] += fi;
      s[1] += fi * VEL[i][0]; s[2] += fi * VEL[i][1]; s[3] += fi * VEL[i][2];
      s[4] += 0.5 * (fi * c2 + g[c * Q + i]);
    }
  }
  for (int k = 0; k < 5; ++k) out5[k] = s[k];
}
