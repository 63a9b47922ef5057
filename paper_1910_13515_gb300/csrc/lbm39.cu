// lbm39.cu -- host runtime of the C ABI declared in include/lbm39.h.
//
// The library owns no device memory: every buffer is the caller's.  Each call
// validates its arguments, enqueues kernels on the lattice's stream and maps
// CUDA errors to LBM39_ERR_CUDA.  Kernels are instantiated for the two
// population storages: double (LBM39_FP64) and float deviations (LBM39_MIXED).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <chrono>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/lbm39.h"
#include "batch.cuh"
#include "kernels.cuh"
#include "lattice_view.h"
#include "prandtl.h"
#include "root_finders.h"

using namespace lbm39;

namespace {

constexpr int BLK = 64;                          // threads per block of the cell kernels
constexpr size_t WS_BYTES = (size_t)BLK * WS_DOUBLES * sizeof(double);
constexpr int RED_BLOCKS = 1024;                 // blocks of the conserved-sum reduction
constexpr int RED_THREADS = 128;
constexpr long long STAGE_CELLS = 1LL << 20;     // host staging chunk (cells)
constexpr uint64_t CKPT_MAGIC = 0x3933424d4c424c31ull;

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// NVTX range over one call of the C ABI, named after the call, so that a
// timeline profiler shows the host side of each call (enqueue, staging
// copies, waits) above the kernels it launched.  Without a profiler attached
// a push and a pop cost a few nanoseconds.
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

struct AuxLayout {
  size_t lam, ctr, heq, href, fstore, partials, result, stage, total;
};

long long plane_stride(long long N) { return (N + 63) / 64 * 64; }

size_t pop_elem(int precision) { return precision == LBM39_MIXED ? sizeof(float) : sizeof(double); }

AuxLayout aux_layout(long long N) {
  const long long Np = plane_stride(N);
  AuxLayout a;
  size_t off = 0;
  a.lam = off; off = align256(off + sizeof(double) * SOLVER_PLANES * Np);
  a.ctr = off; off = align256(off + sizeof(unsigned long long) * 64);
  a.heq = off; off = align256(off + sizeof(double) * 2 * Q);
  a.href = off; off = align256(off + sizeof(double) * 2 * Q);
  a.fstore = off; off = align256(off + sizeof(double) * 2 * Q);
  a.partials = off; off = align256(off + sizeof(double) * 5 * RED_BLOCKS);
  a.result = off; off = align256(off + sizeof(double) * 8);
  a.stage = off; off = align256(off + sizeof(double) * 6 * std::min(N, STAGE_CELLS));
  a.total = off;
  return a;
}

bool params_ok(const lbm39_params* p) {
  if (!p) return false;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return false;
  const long long N = (long long)p->nx * p->ny * p->nz;
  if (N > (1LL << 31) - 64) return false;  // plane stride (N rounded up to 64) stays 32-bit
  if (!(p->gamma > 1.0) || !(p->tau >= 0.5) || !(p->newton_tol > 0.0)) return false;
  if (p->newton_maxit < 1 || p->newton_maxit > 1000 || p->newton_min_upd < 0 ||
      p->init_maxit < 1 || p->init_maxit > 10000)
    return false;
  if (p->precision != LBM39_FP64 && p->precision != LBM39_MIXED) return false;
  if (p->reduce_2d != 0 && p->reduce_2d != 1) return false;
  if (p->precision == LBM39_MIXED && !(p->ref_rho > 0.0 && p->ref_T > 0.0)) return false;
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(p->ref_u[a])) return false;
  if (!(p->prandtl == 0.0 || p->prandtl == 1.0 ||
        (p->prandtl >= 0.01 && p->prandtl <= 100.0 && 2.0 / (p->gamma - 1.0) - D > 0.0)))
    return false;
  // the other root finders serve the FP64 path with the paper's Pr = 1 collision
  if (p->root_finder < 0 || p->root_finder > 3) return false;
  if (p->root_finder != 0 &&
      (p->precision != LBM39_FP64 || !(p->prandtl == 0.0 || p->prandtl == 1.0)))
    return false;
  for (int a = 0; a < 3; ++a) {
    const int n = a == 0 ? p->nx : a == 1 ? p->ny : p->nz;
    if (!p->periodic[a] && n < 7) return false;  // 3 boundary layers per end + fluid
  }
  return true;
}

// 64-bit FNV-1a over a byte range, continued from h.
uint64_t fnv1a(const void* data, size_t n, uint64_t h = 0xcbf29ce484222325ull) {
  const unsigned char* b = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 0x100000001b3ull;
  }
  return h;
}

// Hash of the run parameters a checkpoint's state depends on (everything in
// lbm39_params except the lattice size, stored separately, and the Newton
// budget of lbm39_init).
uint64_t params_hash(const lbm39_params* p) {
  uint64_t h = fnv1a(p->periodic, sizeof p->periodic);
  h = fnv1a(&p->gamma, sizeof p->gamma, h);
  h = fnv1a(&p->tau, sizeof p->tau, h);
  h = fnv1a(&p->kn_sensor, sizeof p->kn_sensor, h);
  h = fnv1a(&p->newton_tol, sizeof p->newton_tol, h);
  h = fnv1a(&p->newton_maxit, sizeof p->newton_maxit, h);
  h = fnv1a(&p->newton_min_upd, sizeof p->newton_min_upd, h);
  h = fnv1a(&p->precision, sizeof p->precision, h);
  h = fnv1a(&p->ref_rho, sizeof p->ref_rho, h);
  h = fnv1a(&p->ref_T, sizeof p->ref_T, h);
  h = fnv1a(&p->rho_inf, sizeof p->rho_inf, h);
  h = fnv1a(p->u_inf, sizeof p->u_inf, h);
  h = fnv1a(&p->T_inf, sizeof p->T_inf, h);
  h = fnv1a(&p->reduce_2d, sizeof p->reduce_2d, h);
  h = fnv1a(&p->prandtl, sizeof p->prandtl, h);
  h = fnv1a(&p->root_finder, sizeof p->root_finder, h);
  h = fnv1a(p->ref_u, sizeof p->ref_u, h);
  return h;
}

}  // namespace

struct lbm39_lattice {
  lbm39_params p;
  long long N = 0, Np = 0, fluid = 0;
  void* pop = nullptr;
  char* aux = nullptr;
  AuxLayout lay{};
  const uint8_t* mask = nullptr;
  bool ghosts = false;  // freestream or outflow cells
  bool fills = false;   // ghosts or solids: the fill kernels run after each pass
  bool mixed = false;
  cudaStream_t stream = nullptr;
  int device = -1;               // the CUDA device current at lbm39_create
  uint64_t mask_hash = 0;        // FNV-1a of the mask bytes (0 without a mask)
  long long t = 0;
  bool initialized = false;
  Desc desc{};
  unsigned long long* ctr() { return reinterpret_cast<unsigned long long*>(aux + lay.ctr); }
  double* stage() { return reinterpret_cast<double*>(aux + lay.stage); }
  size_t pop_bytes() const { return pop_elem(p.precision) * 2 * Q * Np; }
};

#define CUDA_OK(x)                                   \
  do {                                               \
    if ((x) != cudaSuccess) return LBM39_ERR_CUDA;   \
  } while (0)

static int last_launch() { return cudaGetLastError() == cudaSuccess ? LBM39_OK : LBM39_ERR_CUDA; }

// Kernel launches for one storage type.
template <class P>
struct Launch {
  static void step(lbm39_lattice* L, bool odd) {
    L->desc.t = L->t;
    const unsigned grid = (unsigned)((L->N + BLK - 1) / BLK);
    const unsigned fgrid = (unsigned)((L->N + 255) / 256);
    // the reduced (z-mirror) system serves the FP64 path only (see reduction_allowed)
    constexpr bool fp64 = sizeof(P) == 8;
    if (fp64 && L->p.root_finder != 0) {  // other root finders (root_finders.cu)
      launch_step_root_finder(L->desc, odd, L->p.root_finder, L->stream);
      if (L->fills) {
        if (odd) k_fill_odd<P><<<fgrid, 256, 0, L->stream>>>(L->desc);
        else k_fill_even<P><<<fgrid, 256, 0, L->stream>>>(L->desc);
      }
      return;
    }
    if (L->desc.ph.pr_adjust) {  // Prandtl-number adjustment (prandtl.cu)
      launch_step_prandtl(L->desc, odd, !fp64, L->stream);
      if (L->fills) {
        if (odd) k_fill_odd<P><<<fgrid, 256, 0, L->stream>>>(L->desc);
        else k_fill_even<P><<<fgrid, 256, 0, L->stream>>>(L->desc);
      }
      return;
    }
    if (!odd) {
      if (fp64 && L->desc.d2) k_step<false, P, BLK, fp64><<<grid, BLK, WS_BYTES, L->stream>>>(L->desc);
      else k_step<false, P, BLK, false><<<grid, BLK, WS_BYTES, L->stream>>>(L->desc);
      if (L->fills) k_fill_even<P><<<fgrid, 256, 0, L->stream>>>(L->desc);
    } else {
      if (fp64 && L->desc.d2) k_step<true, P, BLK, fp64><<<grid, BLK, WS_BYTES, L->stream>>>(L->desc);
      else k_step<true, P, BLK, false><<<grid, BLK, WS_BYTES, L->stream>>>(L->desc);
      if (L->fills) k_fill_odd<P><<<fgrid, 256, 0, L->stream>>>(L->desc);
    }
  }
  static void init(lbm39_lattice* L, const double* rho, const double* u, long long us,
                   const double* T, long long c0, long long len) {
    const unsigned grid = (unsigned)((len + BLK - 1) / BLK);
    k_init<P, BLK><<<grid, BLK, WS_BYTES, L->stream>>>(L->desc, rho, u, us, T, c0, len,
                                                       L->p.init_maxit);
  }
  static void macros(lbm39_lattice* L, double* rho, double* u, long long us, double* T,
                     double* p, long long c0, long long len) {
    const unsigned grid = (unsigned)((len + 127) / 128);
    if (L->t & 1)
      k_macros<true, P><<<grid, 128, 0, L->stream>>>(L->desc, rho, u, us, T, p, c0, len);
    else
      k_macros<false, P><<<grid, 128, 0, L->stream>>>(L->desc, rho, u, us, T, p, c0, len);
  }
  static void conserved(lbm39_lattice* L, double* partials, unsigned grid) {
    if (L->t & 1)
      k_conserved<true, P, RED_THREADS><<<grid, RED_THREADS, 0, L->stream>>>(L->desc, partials);
    else
      k_conserved<false, P, RED_THREADS><<<grid, RED_THREADS, 0, L->stream>>>(L->desc, partials);
  }
};

extern "C" {

void lbm39_default_params(lbm39_params* p, int32_t nx, int32_t ny, int32_t nz) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->nx = nx; p->ny = ny; p->nz = nz;
  p->periodic[0] = p->periodic[1] = p->periodic[2] = 1;
  p->gamma = 1.4;
  p->tau = 0.6;
  p->kn_sensor = 1;
  p->newton_tol = 1e-12;
  p->newton_maxit = 30;
  p->newton_min_upd = 0;
  p->init_maxit = 200;
  p->precision = LBM39_FP64;
  p->ref_rho = 1.0; p->ref_T = 0.5;
  p->rho_inf = 1.0; p->T_inf = 0.5;
  p->reduce_2d = 1;
  p->prandtl = 1.0;
}

int lbm39_velocities(int32_t* vel, double* w) {
  for (int i = 0; i < Q; ++i) {
    if (vel) { vel[3 * i] = CX[i]; vel[3 * i + 1] = CY[i]; vel[3 * i + 2] = CZ[i]; }
    if (w) w[i] = weight(i);
  }
  return LBM39_OK;
}

int lbm39_query_bytes(const lbm39_params* p, size_t* pop_bytes, size_t* aux_bytes) {
  if (!params_ok(p)) return LBM39_ERR_ARG;
  const long long N = (long long)p->nx * p->ny * p->nz;
  if (pop_bytes) *pop_bytes = pop_elem(p->precision) * 2 * Q * plane_stride(N);
  if (aux_bytes) *aux_bytes = aux_layout(N).total;
  return LBM39_OK;
}

// Validates the mask on the host; counts fluid cells, notes boundary and solid cells.
static int check_mask(const lbm39_params* p, const std::vector<uint8_t>& m, long long* fluid,
                      bool* ghosts, bool* solids) {
  const long long N = (long long)p->nx * p->ny * p->nz;
  const int n[3] = {p->nx, p->ny, p->nz};
  *fluid = 0;
  *ghosts = *solids = false;
  for (long long c = 0; c < N; ++c) {
    const int x = int(c % p->nx), y = int((c / p->nx) % p->ny),
              z = int(c / ((long long)p->nx * p->ny));
    const int q[3] = {x, y, z};
    bool layer = false;
    for (int a = 0; a < 3; ++a)
      if (!p->periodic[a] && (q[a] < 3 || q[a] >= n[a] - 3)) layer = true;
    const uint8_t v = m[c];
    if (v > 3) return LBM39_ERR_MASK;
    if (v == MASK_FLUID) {
      if (layer) return LBM39_ERR_MASK;
      ++*fluid;
    }
    if (v == MASK_SOLID) *solids = true;
    if (v == MASK_FREE || v == MASK_OUT) {
      if (!layer) return LBM39_ERR_MASK;
      *ghosts = true;
    }
    if (v == MASK_OUT) {
      if (p->periodic[0] || !(x < 3 || x >= p->nx - 3)) return LBM39_ERR_MASK;
      const int xc = std::min(std::max(x, 3), p->nx - 4);
      const uint8_t t = m[c + (xc - x)];
      if (t != MASK_FLUID && t != MASK_FREE) return LBM39_ERR_MASK;
    }
  }
  return LBM39_OK;
}

// Equilibrium populations of one state into dev78 (device) and host78.
static int state_equilibrium(const Phys& ph, cudaStream_t s, double rho, const double* u,
                             double T, int maxit, double* dev78, unsigned long long* dfail,
                             double* host78) {
  CUDA_OK(cudaMemsetAsync(dfail, 0, sizeof(unsigned long long), s));
  k_state_equilibrium<BLK><<<1, BLK, WS_BYTES, s>>>(ph, rho, u[0], u[1], u[2], T, dev78, maxit,
                                                     dfail);
  if (last_launch() != LBM39_OK) return LBM39_ERR_CUDA;
  unsigned long long nf = 0;
  CUDA_OK(cudaMemcpyAsync(host78, dev78, sizeof(double) * 2 * Q, cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaMemcpyAsync(&nf, dfail, sizeof nf, cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaStreamSynchronize(s));
  return nf ? LBM39_ERR_NEWTON : LBM39_OK;
}

int lbm39_create(const lbm39_params* p, const int32_t* vel, const double* w, void* pop_buf,
                 void* aux_buf, const uint8_t* mask_dev, void* cuda_stream,
                 lbm39_lattice** out) {
  if (!out) return LBM39_ERR_ARG;
  *out = nullptr;
  if (!params_ok(p) || !vel || !pop_buf || !aux_buf) return LBM39_ERR_ARG;
  if (((uintptr_t)pop_buf & 255) || ((uintptr_t)aux_buf & 255)) return LBM39_ERR_ARG;
  for (int i = 0; i < Q; ++i) {
    if (vel[3 * i] != CX[i] || vel[3 * i + 1] != CY[i] || vel[3 * i + 2] != CZ[i])
      return LBM39_ERR_LATTICE;
    if (w && w[i] != weight(i)) return LBM39_ERR_LATTICE;
  }
  const long long N = (long long)p->nx * p->ny * p->nz;
  const bool all_periodic = p->periodic[0] && p->periodic[1] && p->periodic[2];
  if (!mask_dev && !all_periodic) return LBM39_ERR_MASK;
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  long long fluid = N;
  bool ghosts = false, solids = false;
  uint64_t mask_hash = 0;
  if (mask_dev) {
    std::vector<uint8_t> m(N);
    CUDA_OK(cudaMemcpyAsync(m.data(), mask_dev, N, cudaMemcpyDeviceToHost, stream));
    CUDA_OK(cudaStreamSynchronize(stream));
    const int rc = check_mask(p, m, &fluid, &ghosts, &solids);
    if (rc) return rc;
    mask_hash = fnv1a(m.data(), m.size());
  }
  int device = -1;
  CUDA_OK(cudaGetDevice(&device));
  lbm39_lattice* L = new (std::nothrow) lbm39_lattice;
  if (!L) return LBM39_ERR_ARG;
  L->p = *p;
  L->device = device;
  L->mask_hash = mask_hash;
  L->N = N;
  L->Np = plane_stride(N);
  L->fluid = fluid;
  L->pop = pop_buf;
  L->aux = static_cast<char*>(aux_buf);
  L->lay = aux_layout(N);
  L->mask = mask_dev;
  L->ghosts = ghosts;
  L->fills = ghosts || solids;
  L->mixed = p->precision == LBM39_MIXED;
  L->stream = stream;
  Desc& d = L->desc;
  d.pop = pop_buf;
  d.lam = reinterpret_cast<double*>(L->aux + L->lay.lam);
  d.mask = mask_dev;
  d.ctr = L->ctr();
  d.heq_inf = reinterpret_cast<const double*>(L->aux + L->lay.heq);
  d.href = reinterpret_cast<const double*>(L->aux + L->lay.href);
  d.free_store = L->aux + L->lay.fstore;
  d.N = N;
  d.Np = L->Np;
  d.nx = p->nx; d.ny = p->ny; d.nz = p->nz;
  for (int a = 0; a < 3; ++a) d.per[a] = p->periodic[a] ? 1 : 0;
  const double cv = 1.0 / (p->gamma - 1.0);
  d.ph.tau = p->tau;
  d.ph.cg = 2.0 * cv - D;
  d.ph.inv_2cv = 1.0 / (2.0 * cv);
  d.ph.tol = p->newton_tol;
  d.ph.maxit = p->newton_maxit;
  d.ph.min_upd = p->newton_min_upd;
  d.ph.kn_sensor = p->kn_sensor ? 1 : 0;
  {
    const double alpha[4] = {1.0, 1.05, 1.35, 1.0 / p->tau};  // Eq. (alpha)
    d.ph.pr_adjust = !(p->prandtl == 0.0 || p->prandtl == 1.0);
    for (int b = 0; b < 4; ++b) {
      const double tau_eff = p->tau * (p->kn_sensor ? alpha[b] : 1.0);
      d.ph.omega[b] = 1.0 / tau_eff;
      // Prandtl-number adjustment: the heat flux relaxes with tau2
      const double tau2 = d.ph.pr_adjust ? 0.5 + (tau_eff - 0.5) / p->prandtl : tau_eff;
      d.ph.domega[b] = 1.0 / tau_eff - 1.0 / tau2;
    }
  }
  int rc = LBM39_OK;
  // reference populations of the precision form and their moments
  double href[2 * Q] = {0}, heq[2 * Q] = {0};
  unsigned long long* dfail = L->ctr() + CTR_N;
  if (L->mixed) {
    rc = state_equilibrium(d.ph, stream, p->ref_rho, p->ref_u, p->ref_T, p->init_maxit,
                           reinterpret_cast<double*>(L->aux + L->lay.href), dfail, href);
    if (rc) { delete L; return rc; }
    for (int k = 0; k < 5; ++k) d.mref[k] = 0.0;
    for (int i = 0; i < Q; ++i) {
      d.mref[0] += href[i];
      d.mref[1] += CX[i] * href[i];
      d.mref[2] += CY[i] * href[i];
      d.mref[3] += CZ[i] * href[i];
      d.mref[4] += (CX[i] * CX[i] + CY[i] * CY[i] + CZ[i] * CZ[i]) * href[i] + href[Q + i];
    }
  }
  // far-field equilibrium for freestream cells, in the stored representation
  if (ghosts) {
    rc = state_equilibrium(d.ph, stream, p->rho_inf, p->u_inf, p->T_inf, p->init_maxit,
                           reinterpret_cast<double*>(L->aux + L->lay.heq), dfail, heq);
    if (rc) { delete L; return rc; }
    if (L->mixed) {
      float fs[2 * Q];
      for (int j = 0; j < 2 * Q; ++j) fs[j] = (float)(heq[j] - href[j]);
      if (cudaMemcpyAsync(L->aux + L->lay.fstore, fs, sizeof fs, cudaMemcpyHostToDevice, stream) !=
          cudaSuccess) { delete L; return LBM39_ERR_CUDA; }
    } else if (cudaMemcpyAsync(L->aux + L->lay.fstore, heq, sizeof heq, cudaMemcpyHostToDevice,
                               stream) != cudaSuccess) {
      delete L;
      return LBM39_ERR_CUDA;
    }
  }
  if (cudaStreamSynchronize(stream) != cudaSuccess) { delete L; return LBM39_ERR_CUDA; }
  *out = L;
  return LBM39_OK;
}

// Device address of a host array of `bytes` bytes that kernels may access
// directly -- page-locked and mapped (cudaHostAlloc, cudaHostRegister, pinned
// torch tensors), its first and last byte in one contiguous mapping -- else
// nullptr (pageable memory goes through the staging area).
static void* mapped_host(const void* p, size_t bytes) {
  if (!p || bytes == 0) return nullptr;
  cudaPointerAttributes a{}, b{};
  const char* last = static_cast<const char*>(p) + (bytes - 1);
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess ||
      cudaPointerGetAttributes(&b, last) != cudaSuccess) {
    cudaGetLastError();  // clear the query's error
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || !a.devicePointer ||
      !b.devicePointer)
    return nullptr;
  if (static_cast<const char*>(b.devicePointer) - static_cast<const char*>(a.devicePointer) !=
      (ptrdiff_t)(bytes - 1))
    return nullptr;
  return a.devicePointer;
}

static int init_range(lbm39_lattice* L, const double* rho, const double* u, long long us,
                      const double* T, long long c0, long long len) {
  if (L->mixed) Launch<float>::init(L, rho, u, us, T, c0, len);
  else Launch<double>::init(L, rho, u, us, T, c0, len);
  return last_launch();
}

static int init_begin(lbm39_lattice* L) {
  CUDA_OK(cudaMemsetAsync(L->pop, 0, L->pop_bytes(), L->stream));
  CUDA_OK(cudaMemsetAsync(L->ctr(), 0, sizeof(unsigned long long) * 64, L->stream));
  L->t = 0;
  L->initialized = true;
  return LBM39_OK;
}

// Whether the z-mirror reduction holds: one cell thick in z, far field and
// every initial u_z zero (the init kernel counted cells with u_z != 0), FP64
// path.  The precision form keeps the full system: its FP32 factorisation also
// forms the z-odd pivots and may reject a direction over one of them, which
// the reduced system would not, so the two would not give the same values.
static bool reduction_allowed(const lbm39_lattice* L) {
  return L->p.reduce_2d == 1 && L->p.nz == 1 && L->p.u_inf[2] == 0.0 && !L->mixed &&
         !L->desc.ph.pr_adjust;
}

// After the init kernels: waits for them and fixes the constraint system.
static int init_end(lbm39_lattice* L) {
  unsigned long long asym = 0;
  CUDA_OK(cudaMemcpyAsync(&asym, L->ctr() + CTR_ASYM, sizeof asym, cudaMemcpyDeviceToHost,
                          L->stream));
  CUDA_OK(cudaStreamSynchronize(L->stream));
  L->desc.d2 = reduction_allowed(L) && asym == 0 ? 1 : 0;
  return LBM39_OK;
}

int lbm39_init(lbm39_lattice* L, const double* rho, const double* u, const double* T) {
  const Range range("lbm39_init");
  if (!L || !rho || !u || !T) return LBM39_ERR_ARG;
  int rc = init_begin(L);
  if (rc) return rc;
  rc = init_range(L, rho, u, L->N, T, 0, L->N);
  if (rc) return rc;
  return init_end(L);
}

int lbm39_init_host(lbm39_lattice* L, const double* rho, const double* u, const double* T) {
  const Range range("lbm39_init_host");
  if (!L || !rho || !u || !T) return LBM39_ERR_ARG;
  int rc = init_begin(L);
  if (rc) return rc;
  const size_t nb = sizeof(double) * L->N;
  const void* drho = mapped_host(rho, nb);
  const void* du = mapped_host(u, 3 * nb);
  const void* dT = mapped_host(T, nb);
  if (drho && du && dT) {  // page-locked: the init kernel reads them directly
    rc = init_range(L, static_cast<const double*>(drho), static_cast<const double*>(du), L->N,
                    static_cast<const double*>(dT), 0, L->N);
    if (rc) return rc;
    return init_end(L);
  }
  const long long C = std::min(L->N, STAGE_CELLS);
  double* s = L->stage();
  for (long long c0 = 0; c0 < L->N; c0 += C) {
    const long long n = std::min(C, L->N - c0);
    CUDA_OK(cudaMemcpyAsync(s, rho + c0, sizeof(double) * n, cudaMemcpyHostToDevice, L->stream));
    for (int a = 0; a < 3; ++a)
      CUDA_OK(cudaMemcpyAsync(s + (1 + a) * C, u + a * L->N + c0, sizeof(double) * n,
                              cudaMemcpyHostToDevice, L->stream));
    CUDA_OK(cudaMemcpyAsync(s + 4 * C, T + c0, sizeof(double) * n, cudaMemcpyHostToDevice, L->stream));
    rc = init_range(L, s, s + C, C, s + 4 * C, c0, n);
    if (rc) return rc;
  }
  return init_end(L);
}

int lbm39_step(lbm39_lattice* L, int64_t nsteps) {
  const Range range("lbm39_step");
  if (!L || nsteps < 0) return LBM39_ERR_ARG;
  if (!L->initialized) return LBM39_ERR_STATE;
  for (int64_t s = 0; s < nsteps; ++s) {
    if (L->mixed) Launch<float>::step(L, L->t & 1);
    else Launch<double>::step(L, L->t & 1);
    if (last_launch() != LBM39_OK) return LBM39_ERR_CUDA;
    ++L->t;
  }
  return LBM39_OK;
}

int lbm39_sync(lbm39_lattice* L, int64_t timeout_us, int64_t* failed_cells) {
  const Range range("lbm39_sync");
  if (!L) return LBM39_ERR_ARG;
  cudaEvent_t ev;
  CUDA_OK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  if (cudaEventRecord(ev, L->stream) != cudaSuccess) {
    cudaEventDestroy(ev);
    return LBM39_ERR_CUDA;
  }
  const auto t0 = std::chrono::steady_clock::now();
  cudaError_t q;
  while ((q = cudaEventQuery(ev)) == cudaErrorNotReady) {
    if (timeout_us >= 0 &&
        std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0)
                .count() > timeout_us) {
      cudaEventDestroy(ev);
      return LBM39_ERR_TIMEOUT;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  cudaEventDestroy(ev);
  if (q != cudaSuccess) return LBM39_ERR_CUDA;
  unsigned long long nf = 0;
  CUDA_OK(cudaMemcpyAsync(&nf, L->ctr() + CTR_FAILED, sizeof nf, cudaMemcpyDeviceToHost, L->stream));
  CUDA_OK(cudaStreamSynchronize(L->stream));
  if (failed_cells) *failed_cells = (int64_t)nf;
  return nf ? LBM39_ERR_NEWTON : LBM39_OK;
}

static int read_range(lbm39_lattice* L, double* rho, double* u, long long us, double* T,
                      double* p, long long c0, long long len) {
  if (L->mixed) Launch<float>::macros(L, rho, u, us, T, p, c0, len);
  else Launch<double>::macros(L, rho, u, us, T, p, c0, len);
  return last_launch();
}

int lbm39_read(lbm39_lattice* L, double* rho, double* u, double* T, double* p) {
  const Range range("lbm39_read");
  if (!L) return LBM39_ERR_ARG;
  if (!L->initialized) return LBM39_ERR_STATE;
  return read_range(L, rho, u, L->N, T, p, 0, L->N);
}

int lbm39_read_host(lbm39_lattice* L, double* rho, double* u, double* T, double* p) {
  const Range range("lbm39_read_host");
  if (!L) return LBM39_ERR_ARG;
  if (!L->initialized) return LBM39_ERR_STATE;
  const size_t nb = sizeof(double) * L->N;
  void* drho = rho ? mapped_host(rho, nb) : nullptr;
  void* du = u ? mapped_host(u, 3 * nb) : nullptr;
  void* dT = T ? mapped_host(T, nb) : nullptr;
  void* dp = p ? mapped_host(p, nb) : nullptr;
  if ((!rho || drho) && (!u || du) && (!T || dT) && (!p || dp)) {
    // page-locked: the read-out kernel writes them directly
    const int rc = read_range(L, static_cast<double*>(drho), static_cast<double*>(du), L->N,
                              static_cast<double*>(dT), static_cast<double*>(dp), 0, L->N);
    if (rc) return rc;
    CUDA_OK(cudaStreamSynchronize(L->stream));
    return LBM39_OK;
  }
  const long long C = std::min(L->N, STAGE_CELLS);
  double* s = L->stage();
  for (long long c0 = 0; c0 < L->N; c0 += C) {
    const long long n = std::min(C, L->N - c0);
    int rc = read_range(L, rho ? s : nullptr, u ? s + C : nullptr, C, T ? s + 4 * C : nullptr,
                        p ? s + 5 * C : nullptr, c0, n);
    if (rc) return rc;
    if (rho) CUDA_OK(cudaMemcpyAsync(rho + c0, s, sizeof(double) * n, cudaMemcpyDeviceToHost, L->stream));
    if (u)
      for (int a = 0; a < 3; ++a)
        CUDA_OK(cudaMemcpyAsync(u + a * L->N + c0, s + (1 + a) * C, sizeof(double) * n,
                                cudaMemcpyDeviceToHost, L->stream));
    if (T) CUDA_OK(cudaMemcpyAsync(T + c0, s + 4 * C, sizeof(double) * n, cudaMemcpyDeviceToHost, L->stream));
    if (p) CUDA_OK(cudaMemcpyAsync(p + c0, s + 5 * C, sizeof(double) * n, cudaMemcpyDeviceToHost, L->stream));
    CUDA_OK(cudaStreamSynchronize(L->stream));
  }
  return LBM39_OK;
}

int lbm39_stats(lbm39_lattice* L, lbm39_stats_t* s) {
  const Range range("lbm39_stats");
  if (!L || !s) return LBM39_ERR_ARG;
  if (!L->initialized) return LBM39_ERR_STATE;
  double* partials = reinterpret_cast<double*>(L->aux + L->lay.partials);
  double* result = reinterpret_cast<double*>(L->aux + L->lay.result);
  const unsigned grid =
      (unsigned)std::min<long long>(RED_BLOCKS, (L->N + RED_THREADS - 1) / RED_THREADS);
  if (L->mixed) Launch<float>::conserved(L, partials, grid);
  else Launch<double>::conserved(L, partials, grid);
  k_sum_partials<<<1, 32, 0, L->stream>>>(partials, (int)grid, result);
  if (last_launch() != LBM39_OK) return LBM39_ERR_CUDA;
  unsigned long long c[CTR_N];
  double r5[5];
  CUDA_OK(cudaMemcpyAsync(c, L->ctr(), sizeof c, cudaMemcpyDeviceToHost, L->stream));
  CUDA_OK(cudaMemcpyAsync(r5, result, sizeof r5, cudaMemcpyDeviceToHost, L->stream));
  CUDA_OK(cudaStreamSynchronize(L->stream));
  std::memset(s, 0, sizeof(*s));
  s->time = L->t;
  s->fluid_cells = L->fluid;
  s->failed_cells = (int64_t)c[CTR_FAILED];
  s->newton_updates = (int64_t)c[CTR_UPDATES];
  for (int k = 0; k < 32; ++k) s->newton_hist[k] = (int64_t)c[CTR_HIST + k];
  for (int k = 0; k < 4; ++k) s->eps_hist[k] = (int64_t)c[CTR_EPS + k];
  for (int k = 0; k < 5; ++k) s->conserved[k] = r5[k];
  s->start32_updates = (int64_t)c[CTR_UPD32];
  s->start32_solves = (int64_t)c[CTR_START32];
  return LBM39_OK;
}

size_t lbm39_checkpoint_bytes(const lbm39_lattice* L) {
  if (!L) return 0;
  return 256 + L->pop_bytes() + sizeof(double) * SOLVER_PLANES * L->Np;
}

int lbm39_save(lbm39_lattice* L, void* buf) {
  const Range range("lbm39_save");
  if (!L || !buf) return LBM39_ERR_ARG;
  if (!L->initialized) return LBM39_ERR_STATE;
  uint64_t hdr[32] = {0};
  hdr[0] = CKPT_MAGIC;
  hdr[1] = (uint64_t)L->t;
  hdr[2] = (uint64_t)L->N;
  hdr[3] = (uint64_t)L->p.precision;
  hdr[4] = (uint64_t)L->desc.d2;
  hdr[5] = (uint64_t)L->p.nx;
  hdr[6] = (uint64_t)L->p.ny;
  hdr[7] = (uint64_t)L->p.nz;
  hdr[8] = params_hash(&L->p);
  hdr[9] = L->mask_hash;
  char* b = static_cast<char*>(buf);
  const size_t pb = L->pop_bytes(), lb = sizeof(double) * SOLVER_PLANES * L->Np;
  CUDA_OK(cudaMemcpyAsync(b, hdr, sizeof hdr, cudaMemcpyDefault, L->stream));
  CUDA_OK(cudaMemcpyAsync(b + 256, L->pop, pb, cudaMemcpyDefault, L->stream));
  CUDA_OK(cudaMemcpyAsync(b + 256 + pb, L->desc.lam, lb, cudaMemcpyDefault, L->stream));
  CUDA_OK(cudaStreamSynchronize(L->stream));
  return LBM39_OK;
}

int lbm39_load(lbm39_lattice* L, const void* buf) {
  const Range range("lbm39_load");
  if (!L || !buf) return LBM39_ERR_ARG;
  uint64_t hdr[32];
  const char* b = static_cast<const char*>(buf);
  CUDA_OK(cudaMemcpyAsync(hdr, b, sizeof hdr, cudaMemcpyDefault, L->stream));
  CUDA_OK(cudaStreamSynchronize(L->stream));
  if (hdr[0] != CKPT_MAGIC || hdr[2] != (uint64_t)L->N || hdr[3] != (uint64_t)L->p.precision ||
      hdr[5] != (uint64_t)L->p.nx || hdr[6] != (uint64_t)L->p.ny || hdr[7] != (uint64_t)L->p.nz ||
      hdr[8] != params_hash(&L->p) || hdr[9] != L->mask_hash)
    return LBM39_ERR_ARG;
  const size_t pb = L->pop_bytes(), lb = sizeof(double) * SOLVER_PLANES * L->Np;
  CUDA_OK(cudaMemcpyAsync(L->pop, b + 256, pb, cudaMemcpyDefault, L->stream));
  CUDA_OK(cudaMemcpyAsync(L->desc.lam, b + 256 + pb, lb, cudaMemcpyDefault, L->stream));
  CUDA_OK(cudaMemsetAsync(L->ctr(), 0, sizeof(unsigned long long) * 64, L->stream));
  CUDA_OK(cudaStreamSynchronize(L->stream));
  L->t = (long long)hdr[1];
  L->desc.d2 = hdr[4] == 1 && reduction_allowed(L) ? 1 : 0;
  L->initialized = true;
  return LBM39_OK;
}

int lbm39_selftest_dfma(double* tflops, void* scratch, size_t scratch_bytes, void* cuda_stream) {
  if (!tflops || !scratch) return LBM39_ERR_ARG;
  int dev = 0, sms = 0;
  CUDA_OK(cudaGetDevice(&dev));
  CUDA_OK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int threads = 256, blocks = sms * 8;
  if (scratch_bytes < sizeof(double) * threads * (size_t)blocks) return LBM39_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  cudaEvent_t e0, e1;
  CUDA_OK(cudaEventCreate(&e0));
  CUDA_OK(cudaEventCreate(&e1));
  const int iters = 2048;
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, s);
    k_selftest_dfma<<<blocks, threads, 0, s>>>(static_cast<double*>(scratch), iters, 0.999999, 1e-7);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) { cudaEventDestroy(e0); cudaEventDestroy(e1); return LBM39_ERR_CUDA; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (last_launch() != LBM39_OK) return LBM39_ERR_CUDA;
  const double fmas = (double)blocks * threads * iters * 32.0;
  *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
  return LBM39_OK;
}

int lbm39_selftest_exp(const double* x, double* y, double* ref, int64_t n, void* cuda_stream) {
  if (!x || !y || !ref || n < 0) return LBM39_ERR_ARG;
  if (n == 0) return LBM39_OK;
  const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
  k_selftest_exp<<<grid, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(x, y, ref, n);
  return last_launch();
}

int lbm39_selftest_rcp(const double* x, double* y, double* ref, float* y32, float* ref32,
                       int64_t n, void* cuda_stream) {
  if (!x || !y || !ref || !y32 || !ref32 || n < 0) return LBM39_ERR_ARG;
  if (n == 0) return LBM39_OK;
  const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
  k_selftest_rcp<<<grid, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(x, y, ref, y32, ref32,
                                                                          n);
  return last_launch();
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Serving form: packed steps of many lattices (see include/lbm39.h).

struct lbm39_batch {
  int maxlat = 0;
  long long maxcells = 0, maxtiles = 0, maxftiles = 0;
  int precision = LBM39_FP64;
  int G = 1;
  cudaStream_t stream = nullptr;
  BatchEntry* dE = nullptr;
  Tile* dT = nullptr;
  Tile* dF = nullptr;
  std::vector<BatchEntry> hE;
  std::vector<Tile> hT, hF;
  int nT2 = 0;  // leading tiles of hT whose lattices take the nine-constraint (z-mirror) solve
  std::vector<lbm39_lattice*> lats;
  std::vector<long long> tend;
  cudaGraphExec_t exec = nullptr;
  bool dirty = true;
};

namespace {
struct BatchLayout {
  size_t E, T, F, total;
  long long maxtiles, maxftiles;
};

BatchLayout batch_layout(int maxlat, long long maxcells) {
  BatchLayout b;
  b.maxtiles = (maxcells + BLK - 1) / BLK + maxlat;
  b.maxftiles = (maxcells + 255) / 256 + maxlat;
  size_t off = 0;
  b.E = off; off = align256(off + sizeof(BatchEntry) * maxlat);
  b.T = off; off = align256(off + sizeof(Tile) * b.maxtiles);
  b.F = off; off = align256(off + sizeof(Tile) * b.maxftiles);
  b.total = off;
  return b;
}

template <class P>
int batch_enqueue(lbm39_batch* B, int s) {
  const int nt = (int)B->hT.size(), nf = (int)B->hF.size(), n2 = B->nT2;
  if constexpr (sizeof(P) == 8) {
    if (n2) k_batch_step<P, BLK, true><<<n2, BLK, WS_BYTES, B->stream>>>(B->dE, B->dT, s);
  }
  if (nt > n2)
    k_batch_step<P, BLK, false><<<nt - n2, BLK, WS_BYTES, B->stream>>>(B->dE, B->dT + n2, s);
  if (nf) k_batch_fill<P><<<nf, 256, 0, B->stream>>>(B->dE, B->dF, s);
  return last_launch();
}

int batch_steps(lbm39_batch* B, int n) {
  for (int s = 0; s < n; ++s) {
    const int rc = B->precision == LBM39_MIXED ? batch_enqueue<float>(B, s) : batch_enqueue<double>(B, s);
    if (rc) return rc;
  }
  const int nl = (int)B->hE.size();
  if (nl) k_batch_advance<<<(nl + 127) / 128, 128, 0, B->stream>>>(B->dE, nl, n);
  return last_launch();
}
}  // namespace

extern "C" {

int lbm39_batch_query_bytes(int32_t max_lattices, int64_t max_cells, size_t* bytes) {
  if (max_lattices < 1 || max_cells < 1 || !bytes) return LBM39_ERR_ARG;
  *bytes = batch_layout(max_lattices, max_cells).total;
  return LBM39_OK;
}

int lbm39_batch_create(int32_t max_lattices, int64_t max_cells, int32_t precision,
                       int32_t graph_steps, void* buf, void* cuda_stream, lbm39_batch** out) {
  if (!out) return LBM39_ERR_ARG;
  *out = nullptr;
  if (max_lattices < 1 || max_cells < 1 || graph_steps < 1 || !buf || ((uintptr_t)buf & 255))
    return LBM39_ERR_ARG;
  if (cuda_stream == nullptr) return LBM39_ERR_ARG;  // graphs cannot be captured on the legacy stream
  if (precision != LBM39_FP64 && precision != LBM39_MIXED) return LBM39_ERR_ARG;
  static bool attr = false;
  if (!attr) {
    CUDA_OK(cudaFuncSetAttribute(k_batch_step<double, BLK, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WS_BYTES));
    CUDA_OK(cudaFuncSetAttribute(k_batch_step<double, BLK, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WS_BYTES));
    CUDA_OK(cudaFuncSetAttribute(k_batch_step<float, BLK, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WS_BYTES));
    attr = true;
  }
  lbm39_batch* B = new (std::nothrow) lbm39_batch;
  if (!B) return LBM39_ERR_ARG;
  const BatchLayout lay = batch_layout(max_lattices, max_cells);
  char* b = static_cast<char*>(buf);
  B->maxlat = max_lattices;
  B->maxcells = max_cells;
  B->maxtiles = lay.maxtiles;
  B->maxftiles = lay.maxftiles;
  B->precision = precision;
  B->G = graph_steps;
  B->stream = static_cast<cudaStream_t>(cuda_stream);
  B->dE = reinterpret_cast<BatchEntry*>(b + lay.E);
  B->dT = reinterpret_cast<Tile*>(b + lay.T);
  B->dF = reinterpret_cast<Tile*>(b + lay.F);
  *out = B;
  return LBM39_OK;
}

int lbm39_batch_set(lbm39_batch* B, lbm39_lattice* const* lattices, const int64_t* t_end,
                    int32_t n) {
  const Range range("lbm39_batch_set");
  if (!B || n < 0 || n > B->maxlat || (n > 0 && (!lattices || !t_end))) return LBM39_ERR_ARG;
  long long cells = 0;
  for (int j = 0; j < n; ++j) {
    lbm39_lattice* L = lattices[j];
    if (!L) return LBM39_ERR_ARG;
    if (!L->initialized) return LBM39_ERR_STATE;
    if (L->p.precision != B->precision || t_end[j] < L->t) return LBM39_ERR_ARG;
    // the packed step is the Pr = 1 collision with the Newton solver
    if (L->desc.ph.pr_adjust || L->p.root_finder != 0) return LBM39_ERR_ARG;
    cells += L->N;
  }
  if (cells > B->maxcells) return LBM39_ERR_ARG;
  B->hE.clear(); B->hT.clear(); B->hF.clear(); B->lats.clear(); B->tend.clear();
  std::vector<Tile> full;  // tiles of lattices with the full 13-constraint solve
  for (int j = 0; j < n; ++j) {
    lbm39_lattice* L = lattices[j];
    BatchEntry e;
    e.d = L->desc;
    e.t0 = L->t;
    e.t_end = t_end[j];
    B->hE.push_back(e);
    B->lats.push_back(L);
    B->tend.push_back(t_end[j]);
    // the nine-constraint (z-mirror) tiles first: they take their own instantiation
    std::vector<Tile>& dst = (!L->mixed && L->desc.d2) ? B->hT : full;
    for (long long c = 0; c < L->N; c += BLK) dst.push_back(Tile{j, 0, c});
    if (L->fills)
      for (long long c = 0; c < L->N; c += 256) B->hF.push_back(Tile{j, 0, c});
  }
  B->nT2 = (int)B->hT.size();
  B->hT.insert(B->hT.end(), full.begin(), full.end());
  if ((long long)B->hT.size() > B->maxtiles || (long long)B->hF.size() > B->maxftiles)
    return LBM39_ERR_ARG;
  if (n) {
    CUDA_OK(cudaMemcpyAsync(B->dE, B->hE.data(), sizeof(BatchEntry) * n, cudaMemcpyHostToDevice, B->stream));
    CUDA_OK(cudaMemcpyAsync(B->dT, B->hT.data(), sizeof(Tile) * B->hT.size(), cudaMemcpyHostToDevice, B->stream));
    if (!B->hF.empty())
      CUDA_OK(cudaMemcpyAsync(B->dF, B->hF.data(), sizeof(Tile) * B->hF.size(), cudaMemcpyHostToDevice, B->stream));
  }
  CUDA_OK(cudaStreamSynchronize(B->stream));
  B->dirty = true;
  return LBM39_OK;
}

int lbm39_batch_run(lbm39_batch* B, int64_t nsteps) {
  const Range range("lbm39_batch_run");
  if (!B || nsteps < 0) return LBM39_ERR_ARG;
  if (B->hE.empty() || nsteps == 0) return LBM39_OK;
  int64_t done = 0;
  while (nsteps - done >= B->G) {
    if (B->dirty || !B->exec) {
      if (B->exec) { cudaGraphExecDestroy(B->exec); B->exec = nullptr; }
      cudaGraph_t g = nullptr;
      CUDA_OK(cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal));
      const int rc = batch_steps(B, B->G);
      const cudaError_t ec = cudaStreamEndCapture(B->stream, &g);
      if (rc != LBM39_OK || ec != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return LBM39_ERR_CUDA;
      }
      const cudaError_t ei = cudaGraphInstantiate(&B->exec, g, 0);
      cudaGraphDestroy(g);
      if (ei != cudaSuccess) { B->exec = nullptr; return LBM39_ERR_CUDA; }
      B->dirty = false;
    }
    CUDA_OK(cudaGraphLaunch(B->exec, B->stream));
    done += B->G;
  }
  if (nsteps > done) {
    const int rc = batch_steps(B, (int)(nsteps - done));
    if (rc) return rc;
  }
  for (size_t j = 0; j < B->lats.size(); ++j) {
    B->lats[j]->t = std::min<long long>(B->lats[j]->t + nsteps, B->tend[j]);
    B->hE[j].t0 += nsteps;
  }
  return LBM39_OK;
}

void lbm39_batch_destroy(lbm39_batch* B) {
  if (!B) return;
  if (B->exec) cudaGraphExecDestroy(B->exec);
  delete B;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Conserved sums for callers that cannot allocate device memory.
//
// The reduction's scratch (one partial per block, then the 5 results) is this
// file-scope device array, 320 KiB held by every GPU that loads the library.
// In host code its name is only a stand-in for the device object, so the
// device address is looked up with cudaGetSymbolAddress once per device (on
// the first call with that device current) and handed to the kernels.  Every
// block writes its own partial before the final kernel reads it, so nothing
// has to start at zero; calls that overlap on the GPU share the array and race.
constexpr int NOALLOC_BLOCKS_MAX = 8192;
constexpr int NOALLOC_THREADS = 128;
constexpr long long NOALLOC_CELLS_PER_BLOCK = 8192;  // 64 cells per thread
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_BLOCKS_MAX * 5 + 8];

// Sums over the fluid cells of block b's chunk [b*C, (b+1)*C) into partials[5b..5b+4].
template <bool ODD, class P>
__global__ void __launch_bounds__(NOALLOC_THREADS) k_conserved_chunks(Desc d, double* partials,
                                                                      long long chunk) {
  __shared__ double red[5][NOALLOC_THREADS];
  double acc[5] = {0, 0, 0, 0, 0};
  const long long c0 = (long long)blockIdx.x * chunk;
  const long long c1 = std::min(d.N, c0 + chunk);
  for (long long cell = c0 + threadIdx.x; cell < c1; cell += NOALLOC_THREADS) {
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
  for (int s = NOALLOC_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
#pragma unroll
      for (int k = 0; k < 5; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 5) partials[blockIdx.x * 5 + threadIdx.x] = red[threadIdx.x][0];
}

static double* noalloc_scratch(int* rc) {
  static std::mutex mu;
  static double* ptr[256] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
    *rc = LBM39_ERR_CUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      *rc = LBM39_ERR_CUDA;
      return nullptr;
    }
    ptr[dev] = static_cast<double*>(p);
  }
  *rc = LBM39_OK;
  return ptr[dev];
}

extern "C" {

int lbm39_conserved_noalloc(lbm39_lattice* L, double* sums5) {
  if (!L || !sums5) return LBM39_ERR_ARG;
  if (!L->initialized) return LBM39_ERR_STATE;
  if (L->N > (long long)NOALLOC_BLOCKS_MAX * NOALLOC_CELLS_PER_BLOCK) return LBM39_ERR_ARG;
  int cur = -1;
  CUDA_OK(cudaGetDevice(&cur));
  if (cur != L->device) return LBM39_ERR_ARG;  // the scratch looked up must be the lattice's
  int rc = LBM39_OK;
  double* scratch = noalloc_scratch(&rc);
  if (!scratch) return rc;
  const unsigned grid = (unsigned)((L->N + NOALLOC_CELLS_PER_BLOCK - 1) / NOALLOC_CELLS_PER_BLOCK);
  double* results = scratch + NOALLOC_BLOCKS_MAX * 5;
  const bool odd = L->t & 1;
  if (L->mixed) {
    if (odd) k_conserved_chunks<true, float><<<grid, NOALLOC_THREADS, 0, L->stream>>>(L->desc, scratch, NOALLOC_CELLS_PER_BLOCK);
    else k_conserved_chunks<false, float><<<grid, NOALLOC_THREADS, 0, L->stream>>>(L->desc, scratch, NOALLOC_CELLS_PER_BLOCK);
  } else {
    if (odd) k_conserved_chunks<true, double><<<grid, NOALLOC_THREADS, 0, L->stream>>>(L->desc, scratch, NOALLOC_CELLS_PER_BLOCK);
    else k_conserved_chunks<false, double><<<grid, NOALLOC_THREADS, 0, L->stream>>>(L->desc, scratch, NOALLOC_CELLS_PER_BLOCK);
  }
  k_sum_partials<<<1, 32, 0, L->stream>>>(scratch, (int)grid, results);
  if (last_launch() != LBM39_OK) return LBM39_ERR_CUDA;
  CUDA_OK(cudaMemcpyAsync(sums5, results, sizeof(double) * 5, cudaMemcpyDeviceToHost, L->stream));
  CUDA_OK(cudaStreamSynchronize(L->stream));
  return LBM39_OK;
}

void lbm39_destroy(lbm39_lattice* L) { delete L; }

const char* lbm39_strerror(int status) {
  switch (status) {
    case LBM39_OK: return "ok";
    case LBM39_ERR_ARG: return "invalid argument";
    case LBM39_ERR_CUDA: return "CUDA runtime error";
    case LBM39_ERR_NEWTON: return "Newton solve failed in some cells";
    case LBM39_ERR_TIMEOUT: return "timed out waiting for the GPU";
    case LBM39_ERR_LATTICE: return "velocity or weight table differs from the compiled D3Q39";
    case LBM39_ERR_MASK: return "mask violates the boundary-layer rules";
    case LBM39_ERR_STATE: return "call out of order";
    default: return "unknown status";
  }
}

}  // extern "C"

namespace lbm39 {

bool lattice_view(const lbm39_lattice* L, LatticeView* v) {
  if (!L || !v) return false;
  v->desc = L->desc;
  v->desc.t = L->t;
  v->stream = L->stream;
  v->N = L->N;
  v->mixed = L->mixed;
  v->initialized = L->initialized;
  v->solver = L->p.precision == LBM39_FP64 ? L->p.root_finder : 0;
  return true;
}

}  // namespace lbm39
