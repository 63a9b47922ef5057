// Host build of the CUDA path's polynomial equilibrium (poly_eq.cuh), so that
// its arithmetic can be compared with the oracle on a machine without a GPU.
#include "../paper_1910_13515_gb300/csrc/poly_eq.cuh"

extern "C" void poly_feq_host(const double* rho, const double* u, const double* T, long long n,
                              double* out) {
  for (long long c = 0; c < n; ++c)
    lbm39::poly::feq_cell(rho[c], u[c], u[n + c], u[2 * n + c], T[c], out + 39 * c);
}

extern "C" void poly_velocities_host(int* vel) {
  for (int i = 0; i < lbm39::Q; ++i) {
    vel[3 * i] = lbm39::CX[i];
    vel[3 * i + 1] = lbm39::CY[i];
    vel[3 * i + 2] = lbm39::CZ[i];
  }
}
