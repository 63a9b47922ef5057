/*
 * lbm39_poly.h -- C ABI of the paper's comparison model on the GB300
 * (sm_103a): BGK with a fourth-order polynomial equilibrium on the D3Q39
 * lattice, with a second population set for the extra degrees of freedom.
 *
 * Sec. 5 (Implementation and efficiency) of arXiv:1910.13515 times this model
 * against the 13-moment model (lbm39.h) on a generic subsonic flow.  It names
 * the model without printing it; this library takes the following readings:
 * - f_i^eq is the Hermite expansion of the Maxwellian rho N(u, T I) about the
 *   lattice temperature th = 2/3 (the second moment per axis of the D3Q39
 *   weights, lbm39_velocities), truncated after the fourth order with every
 *   temperature term kept:
 *   f_i^eq = w_i sum_{n<=4} a^(n) : H^(n)(xi_i) / (n! th^n).
 * - g_i^eq = (2 C_v - D) T f_i^eq: the double population of the 13-moment
 *   model (Sec. 3, Eq. discrete-equilibrium-poly), C_v = 1/(gamma - 1).
 * - rho, u and T are the moments of the 13-moment model: rho = sum f,
 *   rho u = sum f xi, sum f|xi|^2 + sum g = rho u^2 + 2 C_v rho T.
 * - Plain BGK: h* = h - (h - h^eq)/tau for f and g alike; in-place
 *   streaming (AA pattern) over shifts of up to 3 cells.
 * - Lattices are periodic along every axis and have no mask.
 *
 * Conventions are those of lbm39.h: x-fastest cell order with at most
 * 2^31 - 64 cells, float64 fields (velocity as 3 planes of N), lattice
 * temperatures, caller-owned device buffers and stream, lbm39_status codes
 * (lbm39_strerror names them), no CPU fallback.  Only the FP64 form exists.
 */
#ifndef LBM39_POLY_H
#define LBM39_POLY_H

#include <stddef.h>
#include <stdint.h>

#include "lbm39.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm39_poly lbm39_poly;

/* Sizes of the two device buffers of a lattice with parameters *p: pop_bytes
 * for the 78 population planes (float64, plane stride N rounded up to 64),
 * aux_bytes for the reduction scratch.  Only nx, ny, nz, periodic, gamma,
 * tau, precision and kn_sensor are read: every axis periodic,
 * precision = LBM39_FP64 and kn_sensor = 0 (plain BGK), else LBM39_ERR_ARG. */
int lbm39_poly_query_bytes(const lbm39_params* p, size_t* pop_bytes, size_t* aux_bytes);

/* Creates a lattice over caller-owned device buffers of at least the queried
 * sizes, 256-byte aligned (LBM39_ERR_ARG otherwise), working on cuda_stream
 * (a cudaStream_t; NULL is the legacy default stream).  No device work. */
int lbm39_poly_create(const lbm39_params* p, void* pop_buf, void* aux_buf, void* cuda_stream,
                      lbm39_poly** out);

/* Enqueues the initial state f = f^eq, g = g^eq of the fields rho, u
 * (3 planes), T: device arrays of N float64, rho > 0 and T > 0 (not
 * checked).  Time is set to 0. */
int lbm39_poly_init(lbm39_poly* L, const double* rho, const double* u, const double* T);

/* Enqueues nsteps >= 0 time steps (per cell: moments, f^eq and g^eq, BGK,
 * streaming).  LBM39_ERR_STATE before lbm39_poly_init. */
int lbm39_poly_step(lbm39_poly* L, int64_t nsteps);

/* Enqueues the macroscopic fields of the current (pre-collision) state into
 * device arrays of N float64: rho, u (3 planes), T and p = rho*T; any may be
 * NULL. */
int lbm39_poly_read(lbm39_poly* L, double* rho, double* u, double* T, double* p);

/* Sums over the lattice (mass, momentum x/y/z, total energy
 * (sum f|xi|^2 + sum g)/2) into sums5 (host memory, 5 float64); waits for the
 * stream.  Deterministic: fixed reduction order. */
int lbm39_poly_conserved(lbm39_poly* L, double* sums5);

/* Time steps taken since lbm39_poly_init (-1 for NULL). */
int64_t lbm39_poly_time(const lbm39_poly* L);

/* Frees the host handle (not the caller's buffers).  NULL is a no-op. */
void lbm39_poly_destroy(lbm39_poly* L);

#ifdef __cplusplus
}
#endif

#endif /* LBM39_POLY_H */
