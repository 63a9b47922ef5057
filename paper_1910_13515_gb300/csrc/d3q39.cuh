// d3q39.cuh -- compile-time D3Q39 lattice for the CUDA kernels.
//
// Velocity set of Sec. 3 (Shan's E^39_{3,7}): (0,0,0), (1,0,0)_FS,
// (+-1,+-1,+-1), (2,0,0)_FS, (2,2,0)_FS, (3,0,0)_FS.  The library orders the
// populations as the rest velocity followed by 19 (xi, -xi) pairs, so
// opp(i) = i+1 for odd i and i-1 for even i > 0.
#pragma once
#include <cstdint>
#include <type_traits>

namespace lbm39 {

constexpr int Q = 39;   // populations per distribution
constexpr int NM = 13;  // constraints of Eq. (13constraints)
constexpr int D = 3;

constexpr int CX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, -1, 1, 2, -2, 0, 0, 0,
                       0, 2, -2, 2, -2, 2, -2, 2, -2, 0, 0, 0, 0, 3, -3, 0, 0, 0, 0};
constexpr int CY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, 1, -1, -1, 1, 1, -1, 0, 0, 2, -2, 0,
                       0, 2, -2, -2, 2, 0, 0, 0, 0, 2, -2, 2, -2, 0, 0, 3, -3, 0, 0};
constexpr int CZ[Q] = {0, 0, 0, 0, 0, 1, -1, 1, -1, -1, 1, 1, -1, 1, -1, 0, 0, 0, 0, 2,
                       -2, 0, 0, 0, 0, 2, -2, -2, 2, 2, -2, -2, 2, 0, 0, 0, 0, 3, -3};

// Device copies for loops with a run-time direction index.
__constant__ int kCX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, -1, 1, 2, -2, 0, 0, 0,
                           0, 2, -2, 2, -2, 2, -2, 2, -2, 0, 0, 0, 0, 3, -3, 0, 0, 0, 0};
__constant__ int kCY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, 1, -1, -1, 1, 1, -1, 0, 0, 2, -2, 0,
                           0, 2, -2, -2, 2, 0, 0, 0, 0, 2, -2, 2, -2, 0, 0, 3, -3, 0, 0};
__constant__ int kCZ[Q] = {0, 0, 0, 0, 0, 1, -1, 1, -1, -1, 1, 1, -1, 1, -1, 0, 0, 0, 0, 2,
                           -2, 0, 0, 0, 0, 2, -2, -2, 2, 2, -2, -2, 2, 0, 0, 0, 0, 3, -3};

constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
constexpr int c2(int i) { return CX[i] * CX[i] + CY[i] * CY[i] + CZ[i] * CZ[i]; }

// Shan's quadrature weights (lattice metadata; the method never uses them).
constexpr double weight(int i) {
  return c2(i) == 0 ? 1.0 / 12.0
       : c2(i) == 1 ? 1.0 / 12.0
       : c2(i) == 3 ? 1.0 / 27.0
       : c2(i) == 4 ? 2.0 / 135.0
       : c2(i) == 8 ? 1.0 / 432.0
                    : 1.0 / 1620.0;
}

// Monomial basis of Eq. (discrete-equilibrium): phi_k(xi_i) for
// k = [1, x, y, z, x^2, y^2, z^2, xy, xz, yz, x|xi|^2, y|xi|^2, z|xi|^2].
constexpr int phi(int k, int i) {
  const int x = CX[i], y = CY[i], z = CZ[i], s = x * x + y * y + z * z;
  return k == 0 ? 1 : k == 1 ? x : k == 2 ? y : k == 3 ? z : k == 4 ? x * x
       : k == 5 ? y * y : k == 6 ? z * z : k == 7 ? x * y : k == 8 ? x * z
       : k == 9 ? y * z : k == 10 ? x * s : k == 11 ? y * s : z * s;
}

// Packed lower-triangle index of a symmetric 13x13 matrix (l <= k).
constexpr int tri(int k, int l) { return k * (k + 1) / 2 + l; }
constexpr int NTRI = NM * (NM + 1) / 2;

// Velocity with the z component reversed.
constexpr int zmirror(int i) {
  for (int j = 0; j < Q; ++j)
    if (CX[j] == CX[i] && CY[j] == CY[i] && CZ[j] == -CZ[i]) return j;
  return i;
}

// Bit i set where velocity i is the first of its z-mirror pair (or its own mirror).
constexpr unsigned long long zmirror_own_mask() {
  unsigned long long m = 0;
  for (int i = 0; i < Q; ++i)
    if (zmirror(i) >= i) m |= 1ull << i;
  return m;
}
constexpr unsigned long long kZOwn = zmirror_own_mask();

// The constraint system solved per cell: all 13 multipliers, or (D2) the nine
// basis functions even in xi_z.  On a lattice one cell thick in z whose
// populations are z-mirror symmetric (u_z = 0 everywhere), the z-odd residuals
// and the couplings of the z-odd multipliers are exact zeros, so those
// multipliers stay exactly zero and leaving them out changes no value.
// (z-even indices 0, 1, 2, 4, 5, 6, 7, 10, 11 by arithmetic: the map is also
// evaluated at run time in device code, where a host array does not exist)
template <bool D2>
struct Sys {
  static constexpr int N = D2 ? 9 : NM;
  static constexpr int idx(int k) { return !D2 ? k : k < 3 ? k : k < 7 ? k + 1 : k + 3; }
};
static_assert(Sys<true>::idx(0) == 0 && Sys<true>::idx(3) == 4 && Sys<true>::idx(6) == 7 &&
                  Sys<true>::idx(7) == 10 && Sys<true>::idx(8) == 11,
              "z-even basis indices");

// Compile-time loop: f(std::integral_constant<int, i>) for i in [B, E).
template <int B, int E, class Fn>
__device__ __forceinline__ void static_for(Fn&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

enum : uint8_t { MASK_FLUID = 0, MASK_SOLID = 1, MASK_FREE = 2, MASK_OUT = 3 };

}  // namespace lbm39
