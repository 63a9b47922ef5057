/*
 * lbm39.h -- C ABI of the GB300 (sm_103a) 13-moment guided-equilibrium
 * double-distribution-function lattice Boltzmann step on D3Q39.
 *
 * Method: Latt, Coreixas, Beny, Parmigiani, "Efficient supersonic flows
 * through high-order guided equilibrium with lattice Boltzmann",
 * arXiv:1910.13515.  Sec. 2 defines the equilibrium (Eq. discrete-equilibrium,
 * Eq. 13constraints, Eq. discrete-equilibrium-poly); Sec. 3 the lattice, the
 * Newton-Raphson solve, BGK collide-and-stream and the Knudsen-number
 * dependent relaxation time (Eq. DeltaAvg, Eq. alpha); Sec. 4 the boundary
 * conditions (freestream equilibrium, first-order outflow, half-way
 * bounce-back); Sec. 5 the per-cell equilibrium step table.
 *
 * Conventions shared by every call
 * - A lattice has nx*ny*nz cells, x fastest: cell = x + nx*(y + ny*z), and
 *   at most 2^31 - 64 cells (larger lattices are rejected with LBM39_ERR_ARG).
 * - Scalar fields are arrays of N = nx*ny*nz float64; velocity fields are 3
 *   consecutive planes of N (u_x, then u_y, then u_z).
 * - Temperatures are lattice temperatures: p = rho*T, c_s = sqrt(gamma*T).
 * - Mask (uint8, N cells, device memory): 0 fluid, 1 solid (half-way
 *   bounce-back), 2 freestream (far-field equilibrium), 3 outflow (copies the
 *   post-collision populations of the cell whose x is clamped into
 *   [3, nx-4]: zero gradient along x).  Codes 2 and 3 may appear only in the
 *   3 outermost layers of a non-periodic axis (3 is the longest lattice
 *   shift), code 3 only along x; those layers may hold no fluid cell; the
 *   cell an outflow cell copies must be fluid or freestream.  A lattice with
 *   no mask (NULL) is all fluid and fully periodic.
 * - Ownership: the caller allocates and frees every device buffer (the
 *   population and auxiliary buffers sized by lbm39_query_bytes, the mask,
 *   the field arrays) and owns the CUDA stream.  The library keeps only a
 *   small host handle.  There is no CPU fallback: every computation runs in
 *   this library's CUDA kernels, and a call on a machine without a usable
 *   GPU returns LBM39_ERR_CUDA.
 * - Errors: every int-returning call returns LBM39_OK (0) or a negative
 *   lbm39_status; nothing is thrown across the ABI.  lbm39_strerror names
 *   the code.  Calls on one lattice are not thread-safe.
 * - Asynchrony: lbm39_step, lbm39_read and lbm39_diag_fields enqueue work on
 *   the lattice's stream and return; lbm39_init, lbm39_sync, lbm39_stats and
 *   the *_host calls wait for it (lbm39_init reads back whether the initial
 *   state allows the z-mirror reduction of lbm39_params.reduce_2d).
 */
#ifndef LBM39_H
#define LBM39_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM39_Q 39  /* discrete velocities of D3Q39 (Sec. 3) */
#define LBM39_NM 13 /* moment constraints / Lagrange multipliers (Eq. 13constraints) */

typedef enum {
  LBM39_OK = 0,
  LBM39_ERR_ARG = -1,     /* NULL pointer, bad size or parameter out of range */
  LBM39_ERR_CUDA = -2,    /* a CUDA runtime call failed (no GPU, bad pointer, ...) */
  LBM39_ERR_NEWTON = -3,  /* some cells failed the Newton solve (counted, see below) */
  LBM39_ERR_TIMEOUT = -4, /* lbm39_sync gave up waiting */
  LBM39_ERR_LATTICE = -5, /* velocity/weight tables differ from the compiled D3Q39 */
  LBM39_ERR_MASK = -6,    /* mask violates the boundary-layer rules above */
  LBM39_ERR_STATE = -7    /* call out of order (e.g. step before init) */
} lbm39_status;

typedef enum {
  LBM39_FP64 = 0, /* populations, moments, Newton and collision in FP64 */
  LBM39_MIXED = 1 /* populations stored in FP32 as deviations from a reference
                     state, collision in FP32; moments and the constraint solve
                     in FP64 (see lbm39_params.ref_rho / ref_u / ref_T) */
} lbm39_precision;

/* Run parameters (Sec. 3).  lbm39_default_params fills the defaults. */
typedef struct {
  int32_t nx, ny, nz;       /* lattice size, each >= 1 */
  int32_t periodic[3];      /* 1 = periodic axis; 0 = 3 boundary layers per end */
  double gamma;             /* heat-capacity ratio, C_v = 1/(gamma-1) (Sec. 2); > 1 */
  double tau;               /* BGK relaxation time tau_f = tau_g (Pr = 1); >= 0.5 */
  int32_t kn_sensor;        /* 1: tau(eps) = tau*alpha(eps) (Eq. alpha); 0: plain BGK */
  double newton_tol;        /* stop when max_k |G_k|/rho < tol (Sec. 5); default 1e-12 */
  int32_t newton_maxit;     /* updates per solve before a cell counts as failed; 30 */
  int32_t newton_min_upd;   /* updates taken even from a converged warm start; 0 */
  int32_t init_maxit;       /* cold-start updates allowed in lbm39_init; 200 */
  int32_t precision;        /* lbm39_precision */
  double ref_rho, ref_T;    /* LBM39_MIXED reference state (rho_bar, T_bar); see ref_u */
  double rho_inf, u_inf[3], T_inf; /* far-field state held by freestream cells */
  int32_t reduce_2d;        /* 1 (default): on a lattice one cell thick in z whose initial
                               u_z and u_inf[2] are all 0, the populations stay mirror
                               symmetric in z, and the FP64 Newton solve uses the nine
                               z-even constraints (the others are exactly zero there):
                               the same values, less work.  0: always all 13.  The
                               precision form always solves all 13. */
  double prandtl;           /* Prandtl number (Sec. 3 leaves its adjustment out: Pr = 1).
                               1 (default) or 0: the paper's BGK collision.  Otherwise a
                               quasi-equilibrium collision with two relaxation times: f
                               relaxes by BGK with tau_eff = tau alpha(eps); g relaxes
                               with tau_eff towards g^eq and, with 1/tau_eff - 1/tau2,
                               towards g^eq_i (1 + c_i . b), c_i = xi_i - u, b = 2 q /
                               ((2 C_v - D) rho T^2), q = (1/2) sum_i c_i (|c_i|^2 f_i +
                               g_i) the heat flux; so the heat flux relaxes with tau2 =
                               1/2 + (tau_eff - 1/2)/Pr and the stress with tau_eff, and
                               Pr = (tau_eff - 1/2)/(tau2 - 1/2).  Mass, momentum and
                               energy are conserved as before.  Range [0.01, 100];
                               needs 2 C_v - D > 0 (gamma < 5/3). */
  int32_t root_finder;      /* solver of the constraint equations in each time step
                               (lbm39_init's cold start always uses Newton):
                               0 (default): Newton-Raphson (Sec. 3);
                               1: chord-Newton hybrid (the Sec. 6 outlook names other
                               root finders): the same stopping rule, polishing step,
                               budget and failure rule, but the direction reuses the
                               LDL^T factor of the last Jacobian formed in the solve
                               while the previous accepted step reduced max|G| by at
                               least 1e-3 (a chord step), else forms J at the current
                               point; a chord step that does not reduce ||G||_2 is
                               replaced by a Newton step from the same point;
                               2: Newton with a single-precision direction: the
                               residual and the update in FP64, the Jacobian and its
                               LDL^T in FP32, same stopping rule; each step contracts
                               the residual by about cond(J) times the FP32 precision;
                               3: 2 after a single-precision start (the precision
                               form's solver): from the cached equilibrium rounded to
                               FP32, Newton steps entirely in FP32 while the FP32
                               residual max|G| is at least 1e-4 (at most 4, each kept
                               only if it lowers max|G|), then 2 from there.
                               1, 2 and 3 converge to the same equilibrium as Newton
                               (the residual that decides convergence is the FP64 one);
                               FP64 path with Pr = 1 only (the precision form always
                               uses 3). */
  double ref_u[3];          /* LBM39_MIXED: velocity of the reference state (default 0).
                               The stored FP32 values are deviations from the 13-moment
                               equilibrium at (ref_rho, ref_u, ref_T).  FP32 resolves a
                               deviation to about 6e-8 of its size, so a population far
                               below its reference value is stored coarsely: a flow that
                               moves as a whole (a far field at Ma 1.5) keeps its
                               populations close to the reference only if the reference
                               moves with it.  The state must lie inside the moment cone
                               (its equilibrium exists), else lbm39_create fails. */
} lbm39_params;

typedef struct lbm39_lattice lbm39_lattice;

/* Counters since lbm39_init, and the current conserved sums. */
typedef struct {
  int64_t time;             /* time steps taken since lbm39_init */
  int64_t fluid_cells;
  int64_t failed_cells;     /* Newton failures summed over cells and steps */
  int64_t newton_updates;   /* Newton updates summed over cells and steps */
  int64_t newton_hist[32];  /* cell-steps by number of updates (31 = 31 or more) */
  int64_t eps_hist[4];      /* cell-steps by alpha branch of Eq. alpha */
  double conserved[5];      /* sums over fluid cells of rho, rho u_x, rho u_y,
                               rho u_z, rho E = (sum f|xi|^2 + sum g)/2 */
  int64_t start32_updates;  /* float steps of single-precision starts (root_finder 3
                               and the precision form), summed over cells and steps;
                               not among newton_updates */
  int64_t start32_solves;   /* cell-steps whose solve kept at least one of them */
} lbm39_stats_t;

/* Fills *p with defaults for an nx*ny*nz fully periodic FP64 lattice
 * (gamma 1.4, tau 0.6, sensor on, tol 1e-12, maxit 30, min_upd 0,
 * init_maxit 200, reference (rho, u, T) = (1, 0, 0.5), far field (1, 0, 0.5),
 * reduce_2d 1, Pr 1, Newton root finder). */
void lbm39_default_params(lbm39_params* p, int32_t nx, int32_t ny, int32_t nz);

/* The compiled D3Q39 velocity set (Sec. 3: (0,0,0), (1,0,0)_FS, (+-1,+-1,+-1),
 * (2,0,0)_FS, (2,2,0)_FS, (3,0,0)_FS) in the library's population order,
 * vel[3*i + d] (host, 39*3 int32), and Shan's E^39_{3,7} weights w[i] (host,
 * 39 float64; lattice metadata only -- the method is quadrature-free, Sec. 2).
 * Either pointer may be NULL.  Population i of a lattice moves by vel[i]. */
int lbm39_velocities(int32_t* vel, double* w);

/* Sizes in bytes of the two device buffers a lattice needs: the populations
 * (39 f and 39 g planes, FP64 or FP32) and the auxiliary buffer (the per-cell
 * solver state carried between steps for the warm start -- the 13 multipliers
 * and the 39 normalised equilibrium values they give, 52 FP64 planes -- counters,
 * reduction scratch and host staging).  Both buffers must be 256-byte aligned. */
int lbm39_query_bytes(const lbm39_params* p, size_t* pop_bytes, size_t* aux_bytes);

/* Creates a lattice over caller-owned device buffers.  vel/w (host) must equal
 * lbm39_velocities' tables (LBM39_ERR_LATTICE otherwise; w may be NULL).
 * mask_dev: device mask of N cells or NULL (all fluid; needs every axis
 * periodic).  The mask is validated (LBM39_ERR_MASK) and must stay unchanged
 * and alive while the lattice exists.  cuda_stream: a cudaStream_t or NULL
 * for the legacy default stream.  *out receives the handle.  The far-field
 * state (with freestream cells) and, for LBM39_MIXED, the reference state
 * must have a 13-moment equilibrium: if their cold-start solve fails, no
 * lattice is created and LBM39_ERR_NEWTON is returned. */
int lbm39_create(const lbm39_params* p, const int32_t* vel, const double* w, void* pop_buf,
                 void* aux_buf, const uint8_t* mask_dev, void* cuda_stream,
                 lbm39_lattice** out);

/* Initial condition (Sec. 3): every fluid cell at its 13-moment equilibrium
 * f = f^eq(rho, u, T), g = (2C_v - D) T f^eq, from a damped cold-start Newton
 * (at most init_maxit updates).  rho, T: N float64; u: 3*N float64; all device
 * pointers.  Resets time and counters.  Cells whose solve fails are counted
 * (see lbm39_sync). */
int lbm39_init(lbm39_lattice* L, const double* rho, const double* u, const double* T);

/* As lbm39_init with host arrays, and waits until the initial state is
 * formed.  Page-locked arrays (cudaHostAlloc, cudaHostRegister, pinned torch
 * tensors; each array one allocation) are read by the init kernel directly;
 * pageable ones are copied through the staging area of the auxiliary buffer. */
int lbm39_init_host(lbm39_lattice* L, const double* rho, const double* u, const double* T);

/* Enqueues nsteps >= 0 time steps (Sec. 3: per fluid cell, macroscopic
 * moments -> Maxwell-Boltzmann targets -> Newton from the previous step's
 * multipliers -> f^eq, g^eq -> eps, alpha -> BGK on f and g -> streaming by
 * shifts of up to 3 cells with the mask rules).  In-place (AA pattern):
 * even and odd steps use two kernels over one population buffer.
 * A cell whose 13 targets lie outside the moment cone of the 39 velocities
 * has no 13-moment equilibrium; its solve fails, and the cell relaxes to the
 * maximum-entropy equilibrium of the five collision invariants instead
 * (conserving mass, momentum and energy), retrying the full solve once every
 * 8 steps.  Each such cell-step counts as a failure (lbm39_sync). */
int lbm39_step(lbm39_lattice* L, int64_t nsteps);

/* Waits for the lattice's stream for at most timeout_us microseconds (< 0:
 * no limit).  *failed_cells (may be NULL) receives the Newton failures
 * since lbm39_init, summed over cells and steps (cell-steps that took the
 * five-invariant fallback equilibrium, see lbm39_step).  Returns
 * LBM39_ERR_TIMEOUT if the work is still running, LBM39_ERR_NEWTON if
 * failed_cells > 0, else LBM39_OK. */
int lbm39_sync(lbm39_lattice* L, int64_t timeout_us, int64_t* failed_cells);

/* Enqueues the macroscopic fields of the current (pre-collision) state:
 * rho, u (3 planes), T and p = rho*T, N float64 each, device pointers; any
 * may be NULL.  Non-fluid cells read 0. */
int lbm39_read(lbm39_lattice* L, double* rho, double* u, double* T, double* p);

/* Enqueues two per-cell fields of the current state into device arrays of N
 * entries: eps (float64), the Knudsen sensor of Eq. DeltaAvg in FP64,
 * (1/39) sum_i |f_i - f_i^eq| / f_i^eq, against the equilibrium the next step
 * relaxes to; n_upd (int32), the Newton updates that step's solve takes from
 * the stored multipliers (with its retry schedule), -1 where the solve fails
 * and the cell takes the fallback.  These are the sensor and iteration maps of
 * the airfoil run (Sec. 4).  Non-fluid cells read 0.  The state, the time and
 * the counters do not change.  LBM39_ERR_STATE before lbm39_init. */
int lbm39_diag_fields(lbm39_lattice* L, double* eps, int32_t* n_upd);

/* As lbm39_read into host arrays; returns when they are written.  Page-locked
 * arrays (each one allocation) are written by the read-out kernel directly;
 * pageable ones through the staging area of the auxiliary buffer. */
int lbm39_read_host(lbm39_lattice* L, double* rho, double* u, double* T, double* p);

/* Waits for the stream and fills *s (counters and conserved sums). */
int lbm39_stats(lbm39_lattice* L, lbm39_stats_t* s);

/* Bytes of a checkpoint (populations, per-cell solver state, time and parity). */
size_t lbm39_checkpoint_bytes(const lbm39_lattice* L);

/* Copies the full state into / from a caller buffer of
 * lbm39_checkpoint_bytes bytes (host or device pointer).  A lattice loaded
 * from a checkpoint continues bit-identically to the one that saved it, also
 * when it is a newly created lattice.  The 256-byte header records the time,
 * the lattice size (nx, ny, nz), the precision, a hash of the run parameters
 * (every lbm39_params field except the size and init_maxit) and a hash of
 * the mask; lbm39_load returns LBM39_ERR_ARG, and changes nothing, unless all
 * of them match the loading lattice. */
int lbm39_save(lbm39_lattice* L, void* buf);
int lbm39_load(lbm39_lattice* L, const void* buf);

/* ---- Serving form: packed steps of many resident lattices ----------------
 * A batch advances up to max_lattices resident lattices (same precision,
 * together at most max_cells cells) with one packed launch per time step: a
 * launch's blocks are tiles of the lattices, each lattice at its own time
 * (own AA parity) and stopping at its own end time, so every lattice gets
 * exactly the arithmetic of lbm39_step.  Runs of graph_steps steps are
 * captured once into a CUDA graph and replayed; the graph is re-captured
 * after lbm39_batch_set.  The batch's device buffer (lbm39_batch_query_bytes)
 * belongs to the caller, like every other buffer.  The caller orders the
 * batch's stream after the lattices' streams (one shared stream does it). */
typedef struct lbm39_batch lbm39_batch;

int lbm39_batch_query_bytes(int32_t max_lattices, int64_t max_cells, size_t* bytes);

/* precision: lbm39_precision of every lattice the batch will hold;
 * graph_steps >= 1: steps per captured graph; buf: device, 256-byte aligned;
 * cuda_stream: a created stream (NULL, the legacy stream, cannot be captured
 * and is rejected with LBM39_ERR_ARG). */
int lbm39_batch_create(int32_t max_lattices, int64_t max_cells, int32_t precision,
                       int32_t graph_steps, void* buf, void* cuda_stream, lbm39_batch** out);

/* Makes lattices[0..n) the resident set; lattice j steps until its time
 * reaches t_end[j] (>= its current time).  Lattices must be initialised, of
 * the batch's precision, with Pr = 1 (lbm39_params.prandtl 1 or 0) and the
 * Newton root finder (other lattices are rejected with LBM39_ERR_ARG), and
 * stay alive while resident.
 * Synchronous. */
int lbm39_batch_set(lbm39_batch* B, lbm39_lattice* const* lattices, const int64_t* t_end,
                    int32_t n);

/* Enqueues nsteps >= 0 packed steps on the batch's stream: each resident
 * lattice advances min(nsteps, t_end - time) steps; lattice times (and so
 * lbm39_read parities) are updated on return. */
int lbm39_batch_run(lbm39_batch* B, int64_t nsteps);

void lbm39_batch_destroy(lbm39_batch* B);

/* Diagnostic: the GPU's FP64 FMA throughput (TFLOP/s, 2 flops per FMA) from a
 * kernel of independent FMA chains on every SM, best of 3 launches timed with
 * CUDA events on cuda_stream -- the ALU roofline of the FP64 step.  scratch:
 * device buffer of at least 8 * 256 * 8 * (number of SMs) bytes.  Synchronous. */
int lbm39_selftest_dfma(double* tflops, void* scratch, size_t scratch_bytes, void* cuda_stream);

/* Diagnostic of the library's FP64 exponential (the table-driven method of
 * Tang, ACM TOMS 15(2) 1989, used for every f^eq evaluation): for n device
 * values x, writes y[i] = that exponential and ref[i] = CUDA's exp(x[i]), so a
 * caller can bound its error.  x, y, ref: device pointers of n float64;
 * cuda_stream as in lbm39_create.  Returns after enqueueing. */
int lbm39_selftest_exp(const double* x, double* y, double* ref, int64_t n, void* cuda_stream);

/* Check of the step's reciprocals (device arrays of n): y[i] = the FP64
 * reciprocal used for 1/rho and the pivots of the Newton solve (Newton's
 * method from the hardware estimate), ref[i] = CUDA's 1.0 / x[i]; y32[i] = the
 * FP32 reciprocal of the Knudsen-sensor screen (rcp.approx.ftz.f32) of
 * (float)x[i], ref32[i] = CUDA's 1.0f / (float)x[i].  Enqueued on cuda_stream.
 * The paper has no counterpart: these are implementation tests. */
int lbm39_selftest_rcp(const double* x, double* y, double* ref, float* y32, float* ref32,
                       int64_t n, void* cuda_stream);

/* Conserved sums (the conserved[] of lbm39_stats_t: mass, momentum x/y/z,
 * total energy over the fluid cells) for callers that cannot allocate device
 * memory -- for instance code that runs where cudaMalloc is unavailable or
 * forbidden, or that must not grow the device footprint after start-up.  The
 * paper has no counterpart: this is a service of the library.  Neither the
 * caller nor the library allocates anything for it: the reduction's scratch
 * is a fixed 320 KiB device array inside the library, present on every GPU
 * that loads the library until the process exits.  The lattice is the input
 * and sums5 (host, 5 float64) the output; the call waits for the lattice's
 * stream.  The first call on a device looks up that array's device address
 * (with the device current), so make it before any stream capture.  Calls
 * share the array: calls that overlap on the GPU race.  Lattices of more than
 * 67,108,864 cells (8192 blocks of 8192 cells) are rejected with
 * LBM39_ERR_ARG, and so is a call made while a device other than the one
 * current at lbm39_create is current.  The block decomposition differs from lbm39_stats', so the
 * sums agree with it to rounding, not bit for bit. */
int lbm39_conserved_noalloc(lbm39_lattice* L, double* sums5);

/* Releases the handle (not the caller's buffers).  NULL is a no-op. */
void lbm39_destroy(lbm39_lattice* L);

/* Static string naming a status code. */
const char* lbm39_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* LBM39_H */
