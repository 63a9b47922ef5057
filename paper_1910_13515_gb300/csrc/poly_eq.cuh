// poly_eq.cuh -- equilibrium of the paper's comparison model (Sec. 5): the
// fourth-order polynomial (Hermite) equilibrium on D3Q39, host and device.
//
// f_i^eq = rho w_i sum_{n<=4} a^(n) : H^(n)(xi_i) / (n! th^n), with th = 2/3
// the second moment per axis of the D3Q39 weights, H^(n) the tensor Hermite
// polynomials of variance th and a^(n) the Hermite coefficients of the
// Maxwellian rho N(u, T I): a^(n) = rho H^(n)(u; -s), s = T - th.  The full
// contractions make the sum a quartic in cu = xi_i . u whose coefficients
// depend on the cell (u2 = |u|^2, s) and on the shell c2 = |xi_i|^2 only:
//
//   P_i = A0 + A1 cu + A2 cu^2 + A3 cu^3 + A4 cu^4,
//   A0 = 1 - (u2 + 3s)/(2 th) + (3 u2^2 + 30 s u2 + 45 s^2)/(24 th^2)
//        + c2 [s/(2 th^2) - s (u2 + 5s)/(4 th^3)] + c2^2 s^2/(8 th^4),
//   A1 = 1/th - (u2 + 5s)/(2 th^2) + c2 s/(2 th^3),
//   A2 = 1/(2 th^2) - (u2 + 7s)/(4 th^3) + c2 s/(4 th^4),
//   A3 = 1/(6 th^3),  A4 = 1/(24 th^4),
//
// (D = 3; e.g. (u u d)_6 : (xi xi d)_6 = 42 cu^2 + 6 u2 c2), and
// f_i^eq = rho w_i P_i.  The pair (xi, -xi) shares cu^2: its even part
// A0 + A2 cu^2 + A4 cu^4 and odd part cu (A1 + A3 cu^2) give both values.
// g_i^eq = (2 C_v - D) T f_i^eq (the double population of Sec. 3).
#pragma once
#include <cmath>
#include <type_traits>

#include "d3q39.cuh"

namespace lbm39 {
namespace poly {

constexpr double TH = 2.0 / 3.0;
constexpr double IT = 1.5;  // 1 / th
constexpr double IT2 = IT * IT, IT3 = IT2 * IT, IT4 = IT2 * IT2;
constexpr double A3 = IT3 / 6.0, A4 = IT4 / 24.0;

// Cell coefficients: A0 = a00 + c2 (a01 + c2 a02), A1 = a10 + c2 a11,
// A2 = a20 + c2 a21.
struct Coef {
  double a00, a01, a02, a10, a11, a20, a21;
};

__host__ __device__ __forceinline__ Coef coefficients(double u2, double s) {
  Coef k;
  k.a00 = 1.0 - (u2 + 3.0 * s) * (0.5 * IT) +
          (3.0 * u2 * u2 + 30.0 * s * u2 + 45.0 * s * s) * (IT2 / 24.0);
  k.a01 = s * (0.5 * IT2) - s * (u2 + 5.0 * s) * (0.25 * IT3);
  k.a02 = s * s * (0.125 * IT4);
  k.a10 = IT - (u2 + 5.0 * s) * (0.5 * IT2);
  k.a11 = s * (0.5 * IT3);
  k.a20 = 0.5 * IT2 - (u2 + 7.0 * s) * (0.25 * IT3);
  k.a21 = s * (0.25 * IT4);
  return k;
}

// The five shell coefficients times a scale W (rho w_i, or omega rho w_i).
struct Shell {
  double b0, b1, b2, b3, b4;
};

template <int C2>
__host__ __device__ __forceinline__ Shell shell(const Coef& k, double W) {
  constexpr double c = C2;
  Shell b;
  b.b0 = W * fma(c, fma(c, k.a02, k.a01), k.a00);
  b.b1 = W * fma(c, k.a11, k.a10);
  b.b2 = W * fma(c, k.a21, k.a20);
  b.b3 = W * A3;
  b.b4 = W * A4;
  return b;
}

// v * C for a small integer C (sign changes exact).
template <int C>
__host__ __device__ __forceinline__ double times(double v) {
  if constexpr (C == 1) return v;
  else if constexpr (C == -1) return -v;
  else return (double)C * v;
}

// xi . u for a constant xi, leaving out its zero components (0 * v does not
// fold away in IEEE arithmetic).
template <int X, int Y, int Z>
__host__ __device__ __forceinline__ double dot(double ux, double uy, double uz) {
  static_assert(X != 0 || Y != 0 || Z != 0, "rest velocity");
  if constexpr (X != 0 && Y != 0 && Z != 0) return times<X>(ux) + times<Y>(uy) + times<Z>(uz);
  else if constexpr (X != 0 && Y != 0) return times<X>(ux) + times<Y>(uy);
  else if constexpr (X != 0 && Z != 0) return times<X>(ux) + times<Z>(uz);
  else if constexpr (Y != 0 && Z != 0) return times<Y>(uy) + times<Z>(uz);
  else if constexpr (X != 0) return times<X>(ux);
  else if constexpr (Y != 0) return times<Y>(uy);
  else return times<Z>(uz);
}

// The scaled equilibrium of the pair (i, i+1) = (xi, -xi), i odd: returns
// W_i P_i in qp and W_i P_{i+1} in qm, W_i = scale * w_i.
template <int I>
__host__ __device__ __forceinline__ void pair_values(const Coef& k, double scale, double ux,
                                                     double uy, double uz, double& qp,
                                                     double& qm) {
  static_assert(I % 2 == 1 && I + 1 < Q, "pairs are (odd i, i + 1)");
  const Shell b = shell<c2(I)>(k, scale * weight(I));
  const double cu = dot<CX[I], CY[I], CZ[I]>(ux, uy, uz);
  const double cu2 = cu * cu;
  const double even = fma(cu2, fma(cu2, b.b4, b.b2), b.b0);
  const double odd = cu * fma(cu2, b.b3, b.b1);
  qp = even + odd;
  qm = even - odd;
}

template <int B, int E, class Fn>
__host__ __device__ __forceinline__ void pairs_for(Fn&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, 2 * B + 1>{});
    pairs_for<B + 1, E>(f);
  }
}

// f^eq of one cell (39 values, library order) from rho, u, T.
__host__ __device__ __forceinline__ void feq_cell(double rho, double ux, double uy, double uz,
                                                  double T, double* out) {
  const Coef k = coefficients(ux * ux + uy * uy + uz * uz, T - TH);
  out[0] = rho * weight(0) * k.a00;
  pairs_for<0, (Q - 1) / 2>([&](auto P) {
    constexpr int i = decltype(P)::value;
    pair_values<i>(k, rho, ux, uy, uz, out[i], out[i + 1]);
  });
}

}  // namespace poly
}  // namespace lbm39
