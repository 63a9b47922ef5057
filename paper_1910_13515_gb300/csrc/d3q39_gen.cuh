// d3q39_gen.cuh -- GENERATED by gen_d3q39.py; do not edit.
#pragma once

namespace lbm39 {
namespace gen {

// Rounded products that are never contracted into a fused multiply-add.
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }

// e_i = sum_k l_k phi_k(xi_i) for every velocity (exponent of Eq. discrete-equilibrium),
// in the type of l (double; float for the single-precision start of a solve).
template <class T>
__device__ __forceinline__ void exponents(const T (&l)[13], T (&e)[39]) {
  const T c0_0 = l[0];
  e[0] = c0_0;
  const T c1_0 = l[0] + l[6];
  const T c1_z = l[3] + l[12];
  const T t1_0_0 = c1_0 + c1_z;
  const T t1_0_1 = c1_0 - c1_z;
  e[5] = t1_0_0;
  e[6] = t1_0_1;
  const T c2_0 = fma(T(4), l[6], l[0]);
  const T c2_z = fma(T(8), l[12], mul_rn(T(2), l[3]));
  const T t2_0_0 = c2_0 + c2_z;
  const T t2_0_1 = c2_0 - c2_z;
  e[19] = t2_0_0;
  e[20] = t2_0_1;
  const T c3_0 = fma(T(9), l[6], l[0]);
  const T c3_z = fma(T(27), l[12], mul_rn(T(3), l[3]));
  const T t3_0_0 = c3_0 + c3_z;
  const T t3_0_1 = c3_0 - c3_z;
  e[37] = t3_0_0;
  e[38] = t3_0_1;
  const T c4_0 = l[0] + l[5];
  const T c4_y = l[2] + l[11];
  const T t4_0_0 = c4_0 + c4_y;
  const T t4_0_1 = c4_0 - c4_y;
  e[3] = t4_0_0;
  e[4] = t4_0_1;
  const T c5_0 = fma(T(4), l[5], l[0]);
  const T c5_y = fma(T(8), l[11], mul_rn(T(2), l[2]));
  const T t5_0_0 = c5_0 + c5_y;
  const T t5_0_1 = c5_0 - c5_y;
  e[17] = t5_0_0;
  e[18] = t5_0_1;
  const T c6_0 = fma(T(4), l[6], fma(T(4), l[5], l[0]));
  const T c6_y = fma(T(16), l[11], mul_rn(T(2), l[2]));
  const T c6_z = fma(T(16), l[12], mul_rn(T(2), l[3]));
  const T c6_yz = mul_rn(T(4), l[9]);
  const T t6_0_0 = c6_0 + c6_y;
  const T t6_0_1 = c6_0 - c6_y;
  const T t6_0_2 = c6_z + c6_yz;
  const T t6_0_3 = c6_z - c6_yz;
  const T t6_1_0 = t6_0_0 + t6_0_2;
  const T t6_1_1 = t6_0_0 - t6_0_2;
  const T t6_1_2 = t6_0_1 + t6_0_3;
  const T t6_1_3 = t6_0_1 - t6_0_3;
  e[29] = t6_1_0;
  e[31] = t6_1_1;
  e[32] = t6_1_2;
  e[30] = t6_1_3;
  const T c7_0 = fma(T(9), l[5], l[0]);
  const T c7_y = fma(T(27), l[11], mul_rn(T(3), l[2]));
  const T t7_0_0 = c7_0 + c7_y;
  const T t7_0_1 = c7_0 - c7_y;
  e[35] = t7_0_0;
  e[36] = t7_0_1;
  const T c8_0 = l[0] + l[4];
  const T c8_x = l[1] + l[10];
  const T t8_0_0 = c8_0 + c8_x;
  const T t8_0_1 = c8_0 - c8_x;
  e[1] = t8_0_0;
  e[2] = t8_0_1;
  const T c9_0 = l[0] + l[4] + l[5] + l[6];
  const T c9_x = fma(T(3), l[10], l[1]);
  const T c9_y = fma(T(3), l[11], l[2]);
  const T c9_z = fma(T(3), l[12], l[3]);
  const T c9_xy = l[7];
  const T c9_xz = l[8];
  const T c9_yz = l[9];
  const T t9_0_0 = c9_0 + c9_x;
  const T t9_0_1 = c9_0 - c9_x;
  const T t9_0_2 = c9_y + c9_xy;
  const T t9_0_3 = c9_y - c9_xy;
  const T t9_0_4 = c9_z + c9_xz;
  const T t9_0_5 = c9_z - c9_xz;
  const T t9_1_0 = t9_0_0 + t9_0_2;
  const T t9_1_1 = t9_0_0 - t9_0_2;
  const T t9_1_2 = t9_0_1 + t9_0_3;
  const T t9_1_3 = t9_0_1 - t9_0_3;
  const T t9_1_4 = t9_0_4 + c9_yz;
  const T t9_1_5 = t9_0_4 - c9_yz;
  const T t9_1_6 = t9_0_5 + c9_yz;
  const T t9_1_7 = t9_0_5 - c9_yz;
  const T t9_2_0 = t9_1_0 + t9_1_4;
  const T t9_2_1 = t9_1_0 - t9_1_4;
  const T t9_2_2 = t9_1_1 + t9_1_5;
  const T t9_2_3 = t9_1_1 - t9_1_5;
  const T t9_2_4 = t9_1_2 + t9_1_6;
  const T t9_2_5 = t9_1_2 - t9_1_6;
  const T t9_2_6 = t9_1_3 + t9_1_7;
  const T t9_2_7 = t9_1_3 - t9_1_7;
  e[7] = t9_2_0;
  e[9] = t9_2_1;
  e[11] = t9_2_2;
  e[14] = t9_2_3;
  e[13] = t9_2_4;
  e[12] = t9_2_5;
  e[10] = t9_2_6;
  e[8] = t9_2_7;
  const T c10_0 = fma(T(4), l[4], l[0]);
  const T c10_x = fma(T(8), l[10], mul_rn(T(2), l[1]));
  const T t10_0_0 = c10_0 + c10_x;
  const T t10_0_1 = c10_0 - c10_x;
  e[15] = t10_0_0;
  e[16] = t10_0_1;
  const T c11_0 = fma(T(4), l[6], fma(T(4), l[4], l[0]));
  const T c11_x = fma(T(16), l[10], mul_rn(T(2), l[1]));
  const T c11_z = fma(T(16), l[12], mul_rn(T(2), l[3]));
  const T c11_xz = mul_rn(T(4), l[8]);
  const T t11_0_0 = c11_0 + c11_x;
  const T t11_0_1 = c11_0 - c11_x;
  const T t11_0_2 = c11_z + c11_xz;
  const T t11_0_3 = c11_z - c11_xz;
  const T t11_1_0 = t11_0_0 + t11_0_2;
  const T t11_1_1 = t11_0_0 - t11_0_2;
  const T t11_1_2 = t11_0_1 + t11_0_3;
  const T t11_1_3 = t11_0_1 - t11_0_3;
  e[25] = t11_1_0;
  e[27] = t11_1_1;
  e[28] = t11_1_2;
  e[26] = t11_1_3;
  const T c12_0 = fma(T(4), l[5], fma(T(4), l[4], l[0]));
  const T c12_x = fma(T(16), l[10], mul_rn(T(2), l[1]));
  const T c12_y = fma(T(16), l[11], mul_rn(T(2), l[2]));
  const T c12_xy = mul_rn(T(4), l[7]);
  const T t12_0_0 = c12_0 + c12_x;
  const T t12_0_1 = c12_0 - c12_x;
  const T t12_0_2 = c12_y + c12_xy;
  const T t12_0_3 = c12_y - c12_xy;
  const T t12_1_0 = t12_0_0 + t12_0_2;
  const T t12_1_1 = t12_0_0 - t12_0_2;
  const T t12_1_2 = t12_0_1 + t12_0_3;
  const T t12_1_3 = t12_0_1 - t12_0_3;
  e[21] = t12_1_0;
  e[23] = t12_1_1;
  e[24] = t12_1_2;
  e[22] = t12_1_3;
  const T c13_0 = fma(T(9), l[4], l[0]);
  const T c13_x = fma(T(27), l[10], mul_rn(T(3), l[1]));
  const T t13_0_0 = c13_0 + c13_x;
  const T t13_0_1 = c13_0 - c13_x;
  e[33] = t13_0_0;
  e[34] = t13_0_1;
}

// The same with the z-odd multipliers zero (lattice one cell thick in z, u_z = 0).
template <class T>
__device__ __forceinline__ void exponents2d(const T (&l)[13], T (&e)[39]) {
  const T c0_0 = l[0];
  e[0] = c0_0;
  const T c1_0 = l[0] + l[6];
  e[5] = c1_0;
  e[6] = c1_0;
  const T c2_0 = fma(T(4), l[6], l[0]);
  e[19] = c2_0;
  e[20] = c2_0;
  const T c3_0 = fma(T(9), l[6], l[0]);
  e[37] = c3_0;
  e[38] = c3_0;
  const T c4_0 = l[0] + l[5];
  const T c4_y = l[2] + l[11];
  const T t4_0_0 = c4_0 + c4_y;
  const T t4_0_1 = c4_0 - c4_y;
  e[3] = t4_0_0;
  e[4] = t4_0_1;
  const T c5_0 = fma(T(4), l[5], l[0]);
  const T c5_y = fma(T(8), l[11], mul_rn(T(2), l[2]));
  const T t5_0_0 = c5_0 + c5_y;
  const T t5_0_1 = c5_0 - c5_y;
  e[17] = t5_0_0;
  e[18] = t5_0_1;
  const T c6_0 = fma(T(4), l[6], fma(T(4), l[5], l[0]));
  const T c6_y = fma(T(16), l[11], mul_rn(T(2), l[2]));
  const T t6_0_0 = c6_0 + c6_y;
  const T t6_0_1 = c6_0 - c6_y;
  e[29] = t6_0_0;
  e[31] = t6_0_0;
  e[32] = t6_0_1;
  e[30] = t6_0_1;
  const T c7_0 = fma(T(9), l[5], l[0]);
  const T c7_y = fma(T(27), l[11], mul_rn(T(3), l[2]));
  const T t7_0_0 = c7_0 + c7_y;
  const T t7_0_1 = c7_0 - c7_y;
  e[35] = t7_0_0;
  e[36] = t7_0_1;
  const T c8_0 = l[0] + l[4];
  const T c8_x = l[1] + l[10];
  const T t8_0_0 = c8_0 + c8_x;
  const T t8_0_1 = c8_0 - c8_x;
  e[1] = t8_0_0;
  e[2] = t8_0_1;
  const T c9_0 = l[0] + l[4] + l[5] + l[6];
  const T c9_x = fma(T(3), l[10], l[1]);
  const T c9_y = fma(T(3), l[11], l[2]);
  const T c9_xy = l[7];
  const T t9_0_0 = c9_0 + c9_x;
  const T t9_0_1 = c9_0 - c9_x;
  const T t9_0_2 = c9_y + c9_xy;
  const T t9_0_3 = c9_y - c9_xy;
  const T t9_1_0 = t9_0_0 + t9_0_2;
  const T t9_1_1 = t9_0_0 - t9_0_2;
  const T t9_1_2 = t9_0_1 + t9_0_3;
  const T t9_1_3 = t9_0_1 - t9_0_3;
  e[7] = t9_1_0;
  e[9] = t9_1_0;
  e[11] = t9_1_1;
  e[14] = t9_1_1;
  e[13] = t9_1_2;
  e[12] = t9_1_2;
  e[10] = t9_1_3;
  e[8] = t9_1_3;
  const T c10_0 = fma(T(4), l[4], l[0]);
  const T c10_x = fma(T(8), l[10], mul_rn(T(2), l[1]));
  const T t10_0_0 = c10_0 + c10_x;
  const T t10_0_1 = c10_0 - c10_x;
  e[15] = t10_0_0;
  e[16] = t10_0_1;
  const T c11_0 = fma(T(4), l[6], fma(T(4), l[4], l[0]));
  const T c11_x = fma(T(16), l[10], mul_rn(T(2), l[1]));
  const T t11_0_0 = c11_0 + c11_x;
  const T t11_0_1 = c11_0 - c11_x;
  e[25] = t11_0_0;
  e[27] = t11_0_0;
  e[28] = t11_0_1;
  e[26] = t11_0_1;
  const T c12_0 = fma(T(4), l[5], fma(T(4), l[4], l[0]));
  const T c12_x = fma(T(16), l[10], mul_rn(T(2), l[1]));
  const T c12_y = fma(T(16), l[11], mul_rn(T(2), l[2]));
  const T c12_xy = mul_rn(T(4), l[7]);
  const T t12_0_0 = c12_0 + c12_x;
  const T t12_0_1 = c12_0 - c12_x;
  const T t12_0_2 = c12_y + c12_xy;
  const T t12_0_3 = c12_y - c12_xy;
  const T t12_1_0 = t12_0_0 + t12_0_2;
  const T t12_1_1 = t12_0_0 - t12_0_2;
  const T t12_1_2 = t12_0_1 + t12_0_3;
  const T t12_1_3 = t12_0_1 - t12_0_3;
  e[21] = t12_1_0;
  e[23] = t12_1_1;
  e[24] = t12_1_2;
  e[22] = t12_1_3;
  const T c13_0 = fma(T(9), l[4], l[0]);
  const T c13_x = fma(T(27), l[10], mul_rn(T(3), l[1]));
  const T t13_0_0 = c13_0 + c13_x;
  const T t13_0_1 = c13_0 - c13_x;
  e[33] = t13_0_0;
  e[34] = t13_0_1;
}

// s_k = sum_i F_i phi_k(xi_i) and J_kl = sum_i F_i phi_k(xi_i) phi_l(xi_i) (l <= k,
// packed) from the Walsh-Hadamard coefficients of the sign orbits.
template <class T, class A>
__device__ __forceinline__ void moments(const A& F, T (&s)[13], T (&J)[91]) {
  const T h000_0 = F[0];
  const T w1_0_0 = F[5] + F[6];
  const T w1_0_1 = F[5] - F[6];
  const T h001_0 = w1_0_0;
  const T h001_z = w1_0_1;
  const T w2_0_0 = F[19] + F[20];
  const T w2_0_1 = F[19] - F[20];
  const T h002_0 = w2_0_0;
  const T h002_z = w2_0_1;
  const T w3_0_0 = F[37] + F[38];
  const T w3_0_1 = F[37] - F[38];
  const T h003_0 = w3_0_0;
  const T h003_z = w3_0_1;
  const T w4_0_0 = F[3] + F[4];
  const T w4_0_1 = F[3] - F[4];
  const T h010_0 = w4_0_0;
  const T h010_y = w4_0_1;
  const T w5_0_0 = F[17] + F[18];
  const T w5_0_1 = F[17] - F[18];
  const T h020_0 = w5_0_0;
  const T h020_y = w5_0_1;
  const T w6_0_0 = F[29] + F[32];
  const T w6_0_1 = F[29] - F[32];
  const T w6_0_2 = F[31] + F[30];
  const T w6_0_3 = F[31] - F[30];
  const T w6_1_0 = w6_0_0 + w6_0_2;
  const T w6_1_1 = w6_0_0 - w6_0_2;
  const T w6_1_2 = w6_0_1 + w6_0_3;
  const T w6_1_3 = w6_0_1 - w6_0_3;
  const T h022_0 = w6_1_0;
  const T h022_z = w6_1_1;
  const T h022_y = w6_1_2;
  const T h022_yz = w6_1_3;
  const T w7_0_0 = F[35] + F[36];
  const T w7_0_1 = F[35] - F[36];
  const T h030_0 = w7_0_0;
  const T h030_y = w7_0_1;
  const T w8_0_0 = F[1] + F[2];
  const T w8_0_1 = F[1] - F[2];
  const T h100_0 = w8_0_0;
  const T h100_x = w8_0_1;
  const T w9_0_0 = F[7] + F[13];
  const T w9_0_1 = F[7] - F[13];
  const T w9_0_2 = F[9] + F[12];
  const T w9_0_3 = F[9] - F[12];
  const T w9_0_4 = F[11] + F[10];
  const T w9_0_5 = F[11] - F[10];
  const T w9_0_6 = F[14] + F[8];
  const T w9_0_7 = F[14] - F[8];
  const T w9_1_0 = w9_0_0 + w9_0_4;
  const T w9_1_1 = w9_0_0 - w9_0_4;
  const T w9_1_2 = w9_0_1 + w9_0_5;
  const T w9_1_3 = w9_0_1 - w9_0_5;
  const T w9_1_4 = w9_0_2 + w9_0_6;
  const T w9_1_5 = w9_0_2 - w9_0_6;
  const T w9_1_6 = w9_0_3 + w9_0_7;
  const T w9_1_7 = w9_0_3 - w9_0_7;
  const T w9_2_0 = w9_1_0 + w9_1_4;
  const T w9_2_1 = w9_1_0 - w9_1_4;
  const T w9_2_2 = w9_1_1 + w9_1_5;
  const T w9_2_3 = w9_1_1 - w9_1_5;
  const T w9_2_4 = w9_1_2 + w9_1_6;
  const T w9_2_5 = w9_1_2 - w9_1_6;
  const T w9_2_6 = w9_1_3 + w9_1_7;
  const T w9_2_7 = w9_1_3 - w9_1_7;
  const T h111_0 = w9_2_0;
  const T h111_z = w9_2_1;
  const T h111_y = w9_2_2;
  const T h111_yz = w9_2_3;
  const T h111_x = w9_2_4;
  const T h111_xz = w9_2_5;
  const T h111_xy = w9_2_6;
  const T h111_xyz = w9_2_7;
  const T w10_0_0 = F[15] + F[16];
  const T w10_0_1 = F[15] - F[16];
  const T h200_0 = w10_0_0;
  const T h200_x = w10_0_1;
  const T w11_0_0 = F[25] + F[28];
  const T w11_0_1 = F[25] - F[28];
  const T w11_0_2 = F[27] + F[26];
  const T w11_0_3 = F[27] - F[26];
  const T w11_1_0 = w11_0_0 + w11_0_2;
  const T w11_1_1 = w11_0_0 - w11_0_2;
  const T w11_1_2 = w11_0_1 + w11_0_3;
  const T w11_1_3 = w11_0_1 - w11_0_3;
  const T h202_0 = w11_1_0;
  const T h202_z = w11_1_1;
  const T h202_x = w11_1_2;
  const T h202_xz = w11_1_3;
  const T w12_0_0 = F[21] + F[24];
  const T w12_0_1 = F[21] - F[24];
  const T w12_0_2 = F[23] + F[22];
  const T w12_0_3 = F[23] - F[22];
  const T w12_1_0 = w12_0_0 + w12_0_2;
  const T w12_1_1 = w12_0_0 - w12_0_2;
  const T w12_1_2 = w12_0_1 + w12_0_3;
  const T w12_1_3 = w12_0_1 - w12_0_3;
  const T h220_0 = w12_1_0;
  const T h220_y = w12_1_1;
  const T h220_x = w12_1_2;
  const T h220_xy = w12_1_3;
  const T w13_0_0 = F[33] + F[34];
  const T w13_0_1 = F[33] - F[34];
  const T h300_0 = w13_0_0;
  const T h300_x = w13_0_1;
  const T M000_0 = (((h000_0 + h010_0 + h100_0 + h220_0) + (h001_0 + h020_0 + h111_0 + h300_0)) + ((h002_0 + h022_0 + h200_0) + (h003_0 + h030_0 + h202_0)));
  const T M001_0 = ((fma(T(2), h022_z, fma(T(2), h002_z, h001_z))) + (fma(T(2), h202_z, fma(T(3), h003_z, h111_z))));
  const T M010_0 = ((fma(T(3), h030_y, fma(T(2), h020_y, h010_y))) + (fma(T(2), h220_y, fma(T(2), h022_y, h111_y))));
  const T M100_0 = ((fma(T(2), h220_x, fma(T(2), h200_x, h100_x))) + (fma(T(3), h300_x, fma(T(2), h202_x, h111_x))));
  const T M002_0 = ((fma(T(4), h022_0, fma(T(4), h002_0, h001_0))) + (fma(T(4), h202_0, fma(T(9), h003_0, h111_0))));
  const T M011_0 = fma(T(4), h022_yz, h111_yz);
  const T M020_0 = ((fma(T(9), h030_0, fma(T(4), h020_0, h010_0))) + (fma(T(4), h220_0, fma(T(4), h022_0, h111_0))));
  const T M101_0 = fma(T(4), h202_xz, h111_xz);
  const T M110_0 = fma(T(4), h220_xy, h111_xy);
  const T M200_0 = ((fma(T(4), h220_0, fma(T(4), h200_0, h100_0))) + (fma(T(9), h300_0, fma(T(4), h202_0, h111_0))));
  const T M003_0 = ((fma(T(8), h022_z, fma(T(8), h002_z, h001_z))) + (fma(T(8), h202_z, fma(T(27), h003_z, h111_z))));
  const T M012_0 = fma(T(8), h022_y, h111_y);
  const T M021_0 = fma(T(8), h022_z, h111_z);
  const T M030_0 = ((fma(T(27), h030_y, fma(T(8), h020_y, h010_y))) + (fma(T(8), h220_y, fma(T(8), h022_y, h111_y))));
  const T M102_0 = fma(T(8), h202_x, h111_x);
  const T M111_0 = h111_xyz;
  const T M120_0 = fma(T(8), h220_x, h111_x);
  const T M201_0 = fma(T(8), h202_z, h111_z);
  const T M210_0 = fma(T(8), h220_y, h111_y);
  const T M300_0 = ((fma(T(8), h220_x, fma(T(8), h200_x, h100_x))) + (fma(T(27), h300_x, fma(T(8), h202_x, h111_x))));
  const T M004_0 = ((fma(T(16), h022_0, fma(T(16), h002_0, h001_0))) + (fma(T(16), h202_0, fma(T(81), h003_0, h111_0))));
  const T M013_0 = fma(T(16), h022_yz, h111_yz);
  const T M022_0 = fma(T(16), h022_0, h111_0);
  const T M031_0 = fma(T(16), h022_yz, h111_yz);
  const T M040_0 = ((fma(T(81), h030_0, fma(T(16), h020_0, h010_0))) + (fma(T(16), h220_0, fma(T(16), h022_0, h111_0))));
  const T M103_0 = fma(T(16), h202_xz, h111_xz);
  const T M112_0 = h111_xy;
  const T M121_0 = h111_xz;
  const T M130_0 = fma(T(16), h220_xy, h111_xy);
  const T M202_0 = fma(T(16), h202_0, h111_0);
  const T M211_0 = h111_yz;
  const T M220_0 = fma(T(16), h220_0, h111_0);
  const T M301_0 = fma(T(16), h202_xz, h111_xz);
  const T M310_0 = fma(T(16), h220_xy, h111_xy);
  const T M400_0 = ((fma(T(16), h220_0, fma(T(16), h200_0, h100_0))) + (fma(T(81), h300_0, fma(T(16), h202_0, h111_0))));
  const T M001_1 = ((fma(T(16), h202_z, fma(T(16), h022_z, fma(T(8), h002_z, h001_z)))) + (fma(T(3), h111_z, mul_rn(T(27), h003_z))));
  const T M010_1 = ((fma(T(16), h220_y, fma(T(27), h030_y, fma(T(8), h020_y, h010_y)))) + (fma(T(3), h111_y, mul_rn(T(16), h022_y))));
  const T M100_1 = ((fma(T(27), h300_x, fma(T(16), h202_x, fma(T(3), h111_x, h100_x)))) + (fma(T(16), h220_x, mul_rn(T(8), h200_x))));
  const T M002_1 = ((fma(T(32), h202_0, fma(T(32), h022_0, fma(T(16), h002_0, h001_0)))) + (fma(T(3), h111_0, mul_rn(T(81), h003_0))));
  const T M011_1 = fma(T(3), h111_yz, mul_rn(T(32), h022_yz));
  const T M020_1 = ((fma(T(32), h220_0, fma(T(81), h030_0, fma(T(16), h020_0, h010_0)))) + (fma(T(3), h111_0, mul_rn(T(32), h022_0))));
  const T M101_1 = fma(T(32), h202_xz, mul_rn(T(3), h111_xz));
  const T M110_1 = fma(T(32), h220_xy, mul_rn(T(3), h111_xy));
  const T M200_1 = ((fma(T(81), h300_0, fma(T(32), h202_0, fma(T(3), h111_0, h100_0)))) + (fma(T(32), h220_0, mul_rn(T(16), h200_0))));
  const T M003_1 = ((fma(T(64), h202_z, fma(T(64), h022_z, fma(T(32), h002_z, h001_z)))) + (fma(T(3), h111_z, mul_rn(T(243), h003_z))));
  const T M012_1 = fma(T(3), h111_y, mul_rn(T(64), h022_y));
  const T M021_1 = fma(T(3), h111_z, mul_rn(T(64), h022_z));
  const T M030_1 = ((fma(T(64), h220_y, fma(T(243), h030_y, fma(T(32), h020_y, h010_y)))) + (fma(T(3), h111_y, mul_rn(T(64), h022_y))));
  const T M102_1 = fma(T(64), h202_x, mul_rn(T(3), h111_x));
  const T M111_1 = mul_rn(T(3), h111_xyz);
  const T M120_1 = fma(T(64), h220_x, mul_rn(T(3), h111_x));
  const T M201_1 = fma(T(64), h202_z, mul_rn(T(3), h111_z));
  const T M210_1 = fma(T(64), h220_y, mul_rn(T(3), h111_y));
  const T M300_1 = ((fma(T(243), h300_x, fma(T(64), h202_x, fma(T(3), h111_x, h100_x)))) + (fma(T(64), h220_x, mul_rn(T(32), h200_x))));
  const T M002_2 = ((fma(T(256), h202_0, fma(T(256), h022_0, fma(T(64), h002_0, h001_0)))) + (fma(T(9), h111_0, mul_rn(T(729), h003_0))));
  const T M011_2 = fma(T(9), h111_yz, mul_rn(T(256), h022_yz));
  const T M020_2 = ((fma(T(256), h220_0, fma(T(729), h030_0, fma(T(64), h020_0, h010_0)))) + (fma(T(9), h111_0, mul_rn(T(256), h022_0))));
  const T M101_2 = fma(T(256), h202_xz, mul_rn(T(9), h111_xz));
  const T M110_2 = fma(T(256), h220_xy, mul_rn(T(9), h111_xy));
  const T M200_2 = ((fma(T(729), h300_0, fma(T(256), h202_0, fma(T(9), h111_0, h100_0)))) + (fma(T(256), h220_0, mul_rn(T(64), h200_0))));
  s[0] = M000_0;
  s[1] = M100_0;
  s[2] = M010_0;
  s[3] = M001_0;
  s[4] = M200_0;
  s[5] = M020_0;
  s[6] = M002_0;
  s[7] = M110_0;
  s[8] = M101_0;
  s[9] = M011_0;
  s[10] = M100_1;
  s[11] = M010_1;
  s[12] = M001_1;
  J[0] = M000_0;
  J[1] = M100_0;
  J[2] = M200_0;
  J[3] = M010_0;
  J[4] = M110_0;
  J[5] = M020_0;
  J[6] = M001_0;
  J[7] = M101_0;
  J[8] = M011_0;
  J[9] = M002_0;
  J[10] = M200_0;
  J[11] = M300_0;
  J[12] = M210_0;
  J[13] = M201_0;
  J[14] = M400_0;
  J[15] = M020_0;
  J[16] = M120_0;
  J[17] = M030_0;
  J[18] = M021_0;
  J[19] = M220_0;
  J[20] = M040_0;
  J[21] = M002_0;
  J[22] = M102_0;
  J[23] = M012_0;
  J[24] = M003_0;
  J[25] = M202_0;
  J[26] = M022_0;
  J[27] = M004_0;
  J[28] = M110_0;
  J[29] = M210_0;
  J[30] = M120_0;
  J[31] = M111_0;
  J[32] = M310_0;
  J[33] = M130_0;
  J[34] = M112_0;
  J[35] = M220_0;
  J[36] = M101_0;
  J[37] = M201_0;
  J[38] = M111_0;
  J[39] = M102_0;
  J[40] = M301_0;
  J[41] = M121_0;
  J[42] = M103_0;
  J[43] = M211_0;
  J[44] = M202_0;
  J[45] = M011_0;
  J[46] = M111_0;
  J[47] = M021_0;
  J[48] = M012_0;
  J[49] = M211_0;
  J[50] = M031_0;
  J[51] = M013_0;
  J[52] = M121_0;
  J[53] = M112_0;
  J[54] = M022_0;
  J[55] = M100_1;
  J[56] = M200_1;
  J[57] = M110_1;
  J[58] = M101_1;
  J[59] = M300_1;
  J[60] = M120_1;
  J[61] = M102_1;
  J[62] = M210_1;
  J[63] = M201_1;
  J[64] = M111_1;
  J[65] = M200_2;
  J[66] = M010_1;
  J[67] = M110_1;
  J[68] = M020_1;
  J[69] = M011_1;
  J[70] = M210_1;
  J[71] = M030_1;
  J[72] = M012_1;
  J[73] = M120_1;
  J[74] = M111_1;
  J[75] = M021_1;
  J[76] = M110_2;
  J[77] = M020_2;
  J[78] = M001_1;
  J[79] = M101_1;
  J[80] = M011_1;
  J[81] = M002_1;
  J[82] = M201_1;
  J[83] = M021_1;
  J[84] = M003_1;
  J[85] = M111_1;
  J[86] = M102_1;
  J[87] = M012_1;
  J[88] = M101_2;
  J[89] = M011_2;
  J[90] = M002_2;
}

// s_k = sum_i F_i phi_k(xi_i) only.
template <class T, class A>
__device__ __forceinline__ void moments_s(const A& F, T (&s)[13]) {
  const T h000_0 = F[0];
  const T w1_0_0 = F[5] + F[6];
  const T w1_0_1 = F[5] - F[6];
  const T h001_0 = w1_0_0;
  const T h001_z = w1_0_1;
  const T w2_0_0 = F[19] + F[20];
  const T w2_0_1 = F[19] - F[20];
  const T h002_0 = w2_0_0;
  const T h002_z = w2_0_1;
  const T w3_0_0 = F[37] + F[38];
  const T w3_0_1 = F[37] - F[38];
  const T h003_0 = w3_0_0;
  const T h003_z = w3_0_1;
  const T w4_0_0 = F[3] + F[4];
  const T w4_0_1 = F[3] - F[4];
  const T h010_0 = w4_0_0;
  const T h010_y = w4_0_1;
  const T w5_0_0 = F[17] + F[18];
  const T w5_0_1 = F[17] - F[18];
  const T h020_0 = w5_0_0;
  const T h020_y = w5_0_1;
  const T w6_0_0 = F[29] + F[32];
  const T w6_0_1 = F[29] - F[32];
  const T w6_0_2 = F[31] + F[30];
  const T w6_0_3 = F[31] - F[30];
  const T w6_1_0 = w6_0_0 + w6_0_2;
  const T w6_1_1 = w6_0_0 - w6_0_2;
  const T w6_1_2 = w6_0_1 + w6_0_3;
  const T w6_1_3 = w6_0_1 - w6_0_3;
  const T h022_0 = w6_1_0;
  const T h022_z = w6_1_1;
  const T h022_y = w6_1_2;
  const T h022_yz = w6_1_3;
  const T w7_0_0 = F[35] + F[36];
  const T w7_0_1 = F[35] - F[36];
  const T h030_0 = w7_0_0;
  const T h030_y = w7_0_1;
  const T w8_0_0 = F[1] + F[2];
  const T w8_0_1 = F[1] - F[2];
  const T h100_0 = w8_0_0;
  const T h100_x = w8_0_1;
  const T w9_0_0 = F[7] + F[13];
  const T w9_0_1 = F[7] - F[13];
  const T w9_0_2 = F[9] + F[12];
  const T w9_0_3 = F[9] - F[12];
  const T w9_0_4 = F[11] + F[10];
  const T w9_0_5 = F[11] - F[10];
  const T w9_0_6 = F[14] + F[8];
  const T w9_0_7 = F[14] - F[8];
  const T w9_1_0 = w9_0_0 + w9_0_4;
  const T w9_1_1 = w9_0_0 - w9_0_4;
  const T w9_1_2 = w9_0_1 + w9_0_5;
  const T w9_1_3 = w9_0_1 - w9_0_5;
  const T w9_1_4 = w9_0_2 + w9_0_6;
  const T w9_1_5 = w9_0_2 - w9_0_6;
  const T w9_1_6 = w9_0_3 + w9_0_7;
  const T w9_1_7 = w9_0_3 - w9_0_7;
  const T w9_2_0 = w9_1_0 + w9_1_4;
  const T w9_2_1 = w9_1_0 - w9_1_4;
  const T w9_2_2 = w9_1_1 + w9_1_5;
  const T w9_2_3 = w9_1_1 - w9_1_5;
  const T w9_2_4 = w9_1_2 + w9_1_6;
  const T w9_2_5 = w9_1_2 - w9_1_6;
  const T w9_2_6 = w9_1_3 + w9_1_7;
  const T w9_2_7 = w9_1_3 - w9_1_7;
  const T h111_0 = w9_2_0;
  const T h111_z = w9_2_1;
  const T h111_y = w9_2_2;
  const T h111_yz = w9_2_3;
  const T h111_x = w9_2_4;
  const T h111_xz = w9_2_5;
  const T h111_xy = w9_2_6;
  const T h111_xyz = w9_2_7;
  const T w10_0_0 = F[15] + F[16];
  const T w10_0_1 = F[15] - F[16];
  const T h200_0 = w10_0_0;
  const T h200_x = w10_0_1;
  const T w11_0_0 = F[25] + F[28];
  const T w11_0_1 = F[25] - F[28];
  const T w11_0_2 = F[27] + F[26];
  const T w11_0_3 = F[27] - F[26];
  const T w11_1_0 = w11_0_0 + w11_0_2;
  const T w11_1_1 = w11_0_0 - w11_0_2;
  const T w11_1_2 = w11_0_1 + w11_0_3;
  const T w11_1_3 = w11_0_1 - w11_0_3;
  const T h202_0 = w11_1_0;
  const T h202_z = w11_1_1;
  const T h202_x = w11_1_2;
  const T h202_xz = w11_1_3;
  const T w12_0_0 = F[21] + F[24];
  const T w12_0_1 = F[21] - F[24];
  const T w12_0_2 = F[23] + F[22];
  const T w12_0_3 = F[23] - F[22];
  const T w12_1_0 = w12_0_0 + w12_0_2;
  const T w12_1_1 = w12_0_0 - w12_0_2;
  const T w12_1_2 = w12_0_1 + w12_0_3;
  const T w12_1_3 = w12_0_1 - w12_0_3;
  const T h220_0 = w12_1_0;
  const T h220_y = w12_1_1;
  const T h220_x = w12_1_2;
  const T h220_xy = w12_1_3;
  const T w13_0_0 = F[33] + F[34];
  const T w13_0_1 = F[33] - F[34];
  const T h300_0 = w13_0_0;
  const T h300_x = w13_0_1;
  const T M000_0 = (((h000_0 + h010_0 + h100_0 + h220_0) + (h001_0 + h020_0 + h111_0 + h300_0)) + ((h002_0 + h022_0 + h200_0) + (h003_0 + h030_0 + h202_0)));
  const T M001_0 = ((fma(T(2), h022_z, fma(T(2), h002_z, h001_z))) + (fma(T(2), h202_z, fma(T(3), h003_z, h111_z))));
  const T M010_0 = ((fma(T(3), h030_y, fma(T(2), h020_y, h010_y))) + (fma(T(2), h220_y, fma(T(2), h022_y, h111_y))));
  const T M100_0 = ((fma(T(2), h220_x, fma(T(2), h200_x, h100_x))) + (fma(T(3), h300_x, fma(T(2), h202_x, h111_x))));
  const T M002_0 = ((fma(T(4), h022_0, fma(T(4), h002_0, h001_0))) + (fma(T(4), h202_0, fma(T(9), h003_0, h111_0))));
  const T M011_0 = fma(T(4), h022_yz, h111_yz);
  const T M020_0 = ((fma(T(9), h030_0, fma(T(4), h020_0, h010_0))) + (fma(T(4), h220_0, fma(T(4), h022_0, h111_0))));
  const T M101_0 = fma(T(4), h202_xz, h111_xz);
  const T M110_0 = fma(T(4), h220_xy, h111_xy);
  const T M200_0 = ((fma(T(4), h220_0, fma(T(4), h200_0, h100_0))) + (fma(T(9), h300_0, fma(T(4), h202_0, h111_0))));
  const T M001_1 = ((fma(T(16), h202_z, fma(T(16), h022_z, fma(T(8), h002_z, h001_z)))) + (fma(T(3), h111_z, mul_rn(T(27), h003_z))));
  const T M010_1 = ((fma(T(16), h220_y, fma(T(27), h030_y, fma(T(8), h020_y, h010_y)))) + (fma(T(3), h111_y, mul_rn(T(16), h022_y))));
  const T M100_1 = ((fma(T(27), h300_x, fma(T(16), h202_x, fma(T(3), h111_x, h100_x)))) + (fma(T(16), h220_x, mul_rn(T(8), h200_x))));
  s[0] = M000_0;
  s[1] = M100_0;
  s[2] = M010_0;
  s[3] = M001_0;
  s[4] = M200_0;
  s[5] = M020_0;
  s[6] = M002_0;
  s[7] = M110_0;
  s[8] = M101_0;
  s[9] = M011_0;
  s[10] = M100_1;
  s[11] = M010_1;
  s[12] = M001_1;
}

// z-mirror-symmetric F: s and J of the nine z-even basis functions (ZEVEN order).
template <class T, class A>
__device__ __forceinline__ void moments2d(const A& F, T (&s)[9], T (&J)[45]) {
  const T h000_0 = F[0];
  const T w1_0_0 = F[5] + F[6];
  const T w1_0_1 = F[5] - F[6];
  const T h001_0 = w1_0_0;
  const T h001_z = w1_0_1;
  const T w2_0_0 = F[19] + F[20];
  const T w2_0_1 = F[19] - F[20];
  const T h002_0 = w2_0_0;
  const T h002_z = w2_0_1;
  const T w3_0_0 = F[37] + F[38];
  const T w3_0_1 = F[37] - F[38];
  const T h003_0 = w3_0_0;
  const T h003_z = w3_0_1;
  const T w4_0_0 = F[3] + F[4];
  const T w4_0_1 = F[3] - F[4];
  const T h010_0 = w4_0_0;
  const T h010_y = w4_0_1;
  const T w5_0_0 = F[17] + F[18];
  const T w5_0_1 = F[17] - F[18];
  const T h020_0 = w5_0_0;
  const T h020_y = w5_0_1;
  const T w6_0_0 = F[29] + F[32];
  const T w6_0_1 = F[29] - F[32];
  const T w6_0_2 = F[31] + F[30];
  const T w6_0_3 = F[31] - F[30];
  const T w6_1_0 = w6_0_0 + w6_0_2;
  const T w6_1_1 = w6_0_0 - w6_0_2;
  const T w6_1_2 = w6_0_1 + w6_0_3;
  const T w6_1_3 = w6_0_1 - w6_0_3;
  const T h022_0 = w6_1_0;
  const T h022_z = w6_1_1;
  const T h022_y = w6_1_2;
  const T h022_yz = w6_1_3;
  const T w7_0_0 = F[35] + F[36];
  const T w7_0_1 = F[35] - F[36];
  const T h030_0 = w7_0_0;
  const T h030_y = w7_0_1;
  const T w8_0_0 = F[1] + F[2];
  const T w8_0_1 = F[1] - F[2];
  const T h100_0 = w8_0_0;
  const T h100_x = w8_0_1;
  const T w9_0_0 = F[7] + F[13];
  const T w9_0_1 = F[7] - F[13];
  const T w9_0_2 = F[9] + F[12];
  const T w9_0_3 = F[9] - F[12];
  const T w9_0_4 = F[11] + F[10];
  const T w9_0_5 = F[11] - F[10];
  const T w9_0_6 = F[14] + F[8];
  const T w9_0_7 = F[14] - F[8];
  const T w9_1_0 = w9_0_0 + w9_0_4;
  const T w9_1_1 = w9_0_0 - w9_0_4;
  const T w9_1_2 = w9_0_1 + w9_0_5;
  const T w9_1_3 = w9_0_1 - w9_0_5;
  const T w9_1_4 = w9_0_2 + w9_0_6;
  const T w9_1_5 = w9_0_2 - w9_0_6;
  const T w9_1_6 = w9_0_3 + w9_0_7;
  const T w9_1_7 = w9_0_3 - w9_0_7;
  const T w9_2_0 = w9_1_0 + w9_1_4;
  const T w9_2_1 = w9_1_0 - w9_1_4;
  const T w9_2_2 = w9_1_1 + w9_1_5;
  const T w9_2_3 = w9_1_1 - w9_1_5;
  const T w9_2_4 = w9_1_2 + w9_1_6;
  const T w9_2_5 = w9_1_2 - w9_1_6;
  const T w9_2_6 = w9_1_3 + w9_1_7;
  const T w9_2_7 = w9_1_3 - w9_1_7;
  const T h111_0 = w9_2_0;
  const T h111_z = w9_2_1;
  const T h111_y = w9_2_2;
  const T h111_yz = w9_2_3;
  const T h111_x = w9_2_4;
  const T h111_xz = w9_2_5;
  const T h111_xy = w9_2_6;
  const T h111_xyz = w9_2_7;
  const T w10_0_0 = F[15] + F[16];
  const T w10_0_1 = F[15] - F[16];
  const T h200_0 = w10_0_0;
  const T h200_x = w10_0_1;
  const T w11_0_0 = F[25] + F[28];
  const T w11_0_1 = F[25] - F[28];
  const T w11_0_2 = F[27] + F[26];
  const T w11_0_3 = F[27] - F[26];
  const T w11_1_0 = w11_0_0 + w11_0_2;
  const T w11_1_1 = w11_0_0 - w11_0_2;
  const T w11_1_2 = w11_0_1 + w11_0_3;
  const T w11_1_3 = w11_0_1 - w11_0_3;
  const T h202_0 = w11_1_0;
  const T h202_z = w11_1_1;
  const T h202_x = w11_1_2;
  const T h202_xz = w11_1_3;
  const T w12_0_0 = F[21] + F[24];
  const T w12_0_1 = F[21] - F[24];
  const T w12_0_2 = F[23] + F[22];
  const T w12_0_3 = F[23] - F[22];
  const T w12_1_0 = w12_0_0 + w12_0_2;
  const T w12_1_1 = w12_0_0 - w12_0_2;
  const T w12_1_2 = w12_0_1 + w12_0_3;
  const T w12_1_3 = w12_0_1 - w12_0_3;
  const T h220_0 = w12_1_0;
  const T h220_y = w12_1_1;
  const T h220_x = w12_1_2;
  const T h220_xy = w12_1_3;
  const T w13_0_0 = F[33] + F[34];
  const T w13_0_1 = F[33] - F[34];
  const T h300_0 = w13_0_0;
  const T h300_x = w13_0_1;
  const T M000_0 = (((h000_0 + h010_0 + h100_0 + h220_0) + (h001_0 + h020_0 + h111_0 + h300_0)) + ((h002_0 + h022_0 + h200_0) + (h003_0 + h030_0 + h202_0)));
  const T M010_0 = ((fma(T(3), h030_y, fma(T(2), h020_y, h010_y))) + (fma(T(2), h220_y, fma(T(2), h022_y, h111_y))));
  const T M100_0 = ((fma(T(2), h220_x, fma(T(2), h200_x, h100_x))) + (fma(T(3), h300_x, fma(T(2), h202_x, h111_x))));
  const T M002_0 = ((fma(T(4), h022_0, fma(T(4), h002_0, h001_0))) + (fma(T(4), h202_0, fma(T(9), h003_0, h111_0))));
  const T M020_0 = ((fma(T(9), h030_0, fma(T(4), h020_0, h010_0))) + (fma(T(4), h220_0, fma(T(4), h022_0, h111_0))));
  const T M110_0 = fma(T(4), h220_xy, h111_xy);
  const T M200_0 = ((fma(T(4), h220_0, fma(T(4), h200_0, h100_0))) + (fma(T(9), h300_0, fma(T(4), h202_0, h111_0))));
  const T M012_0 = fma(T(8), h022_y, h111_y);
  const T M030_0 = ((fma(T(27), h030_y, fma(T(8), h020_y, h010_y))) + (fma(T(8), h220_y, fma(T(8), h022_y, h111_y))));
  const T M102_0 = fma(T(8), h202_x, h111_x);
  const T M120_0 = fma(T(8), h220_x, h111_x);
  const T M210_0 = fma(T(8), h220_y, h111_y);
  const T M300_0 = ((fma(T(8), h220_x, fma(T(8), h200_x, h100_x))) + (fma(T(27), h300_x, fma(T(8), h202_x, h111_x))));
  const T M004_0 = ((fma(T(16), h022_0, fma(T(16), h002_0, h001_0))) + (fma(T(16), h202_0, fma(T(81), h003_0, h111_0))));
  const T M022_0 = fma(T(16), h022_0, h111_0);
  const T M040_0 = ((fma(T(81), h030_0, fma(T(16), h020_0, h010_0))) + (fma(T(16), h220_0, fma(T(16), h022_0, h111_0))));
  const T M112_0 = h111_xy;
  const T M130_0 = fma(T(16), h220_xy, h111_xy);
  const T M202_0 = fma(T(16), h202_0, h111_0);
  const T M220_0 = fma(T(16), h220_0, h111_0);
  const T M310_0 = fma(T(16), h220_xy, h111_xy);
  const T M400_0 = ((fma(T(16), h220_0, fma(T(16), h200_0, h100_0))) + (fma(T(81), h300_0, fma(T(16), h202_0, h111_0))));
  const T M010_1 = ((fma(T(16), h220_y, fma(T(27), h030_y, fma(T(8), h020_y, h010_y)))) + (fma(T(3), h111_y, mul_rn(T(16), h022_y))));
  const T M100_1 = ((fma(T(27), h300_x, fma(T(16), h202_x, fma(T(3), h111_x, h100_x)))) + (fma(T(16), h220_x, mul_rn(T(8), h200_x))));
  const T M020_1 = ((fma(T(32), h220_0, fma(T(81), h030_0, fma(T(16), h020_0, h010_0)))) + (fma(T(3), h111_0, mul_rn(T(32), h022_0))));
  const T M110_1 = fma(T(32), h220_xy, mul_rn(T(3), h111_xy));
  const T M200_1 = ((fma(T(81), h300_0, fma(T(32), h202_0, fma(T(3), h111_0, h100_0)))) + (fma(T(32), h220_0, mul_rn(T(16), h200_0))));
  const T M012_1 = fma(T(3), h111_y, mul_rn(T(64), h022_y));
  const T M030_1 = ((fma(T(64), h220_y, fma(T(243), h030_y, fma(T(32), h020_y, h010_y)))) + (fma(T(3), h111_y, mul_rn(T(64), h022_y))));
  const T M102_1 = fma(T(64), h202_x, mul_rn(T(3), h111_x));
  const T M120_1 = fma(T(64), h220_x, mul_rn(T(3), h111_x));
  const T M210_1 = fma(T(64), h220_y, mul_rn(T(3), h111_y));
  const T M300_1 = ((fma(T(243), h300_x, fma(T(64), h202_x, fma(T(3), h111_x, h100_x)))) + (fma(T(64), h220_x, mul_rn(T(32), h200_x))));
  const T M020_2 = ((fma(T(256), h220_0, fma(T(729), h030_0, fma(T(64), h020_0, h010_0)))) + (fma(T(9), h111_0, mul_rn(T(256), h022_0))));
  const T M110_2 = fma(T(256), h220_xy, mul_rn(T(9), h111_xy));
  const T M200_2 = ((fma(T(729), h300_0, fma(T(256), h202_0, fma(T(9), h111_0, h100_0)))) + (fma(T(256), h220_0, mul_rn(T(64), h200_0))));
  s[0] = M000_0;
  s[1] = M100_0;
  s[2] = M010_0;
  s[3] = M200_0;
  s[4] = M020_0;
  s[5] = M002_0;
  s[6] = M110_0;
  s[7] = M100_1;
  s[8] = M010_1;
  J[0] = M000_0;
  J[1] = M100_0;
  J[2] = M200_0;
  J[3] = M010_0;
  J[4] = M110_0;
  J[5] = M020_0;
  J[6] = M200_0;
  J[7] = M300_0;
  J[8] = M210_0;
  J[9] = M400_0;
  J[10] = M020_0;
  J[11] = M120_0;
  J[12] = M030_0;
  J[13] = M220_0;
  J[14] = M040_0;
  J[15] = M002_0;
  J[16] = M102_0;
  J[17] = M012_0;
  J[18] = M202_0;
  J[19] = M022_0;
  J[20] = M004_0;
  J[21] = M110_0;
  J[22] = M210_0;
  J[23] = M120_0;
  J[24] = M310_0;
  J[25] = M130_0;
  J[26] = M112_0;
  J[27] = M220_0;
  J[28] = M100_1;
  J[29] = M200_1;
  J[30] = M110_1;
  J[31] = M300_1;
  J[32] = M120_1;
  J[33] = M102_1;
  J[34] = M210_1;
  J[35] = M200_2;
  J[36] = M010_1;
  J[37] = M110_1;
  J[38] = M020_1;
  J[39] = M210_1;
  J[40] = M030_1;
  J[41] = M012_1;
  J[42] = M120_1;
  J[43] = M110_2;
  J[44] = M020_2;
}

template <class T, class A>
__device__ __forceinline__ void moments_s2d(const A& F, T (&s)[9]) {
  const T h000_0 = F[0];
  const T w1_0_0 = F[5] + F[6];
  const T w1_0_1 = F[5] - F[6];
  const T h001_0 = w1_0_0;
  const T h001_z = w1_0_1;
  const T w2_0_0 = F[19] + F[20];
  const T w2_0_1 = F[19] - F[20];
  const T h002_0 = w2_0_0;
  const T h002_z = w2_0_1;
  const T w3_0_0 = F[37] + F[38];
  const T w3_0_1 = F[37] - F[38];
  const T h003_0 = w3_0_0;
  const T h003_z = w3_0_1;
  const T w4_0_0 = F[3] + F[4];
  const T w4_0_1 = F[3] - F[4];
  const T h010_0 = w4_0_0;
  const T h010_y = w4_0_1;
  const T w5_0_0 = F[17] + F[18];
  const T w5_0_1 = F[17] - F[18];
  const T h020_0 = w5_0_0;
  const T h020_y = w5_0_1;
  const T w6_0_0 = F[29] + F[32];
  const T w6_0_1 = F[29] - F[32];
  const T w6_0_2 = F[31] + F[30];
  const T w6_0_3 = F[31] - F[30];
  const T w6_1_0 = w6_0_0 + w6_0_2;
  const T w6_1_1 = w6_0_0 - w6_0_2;
  const T w6_1_2 = w6_0_1 + w6_0_3;
  const T w6_1_3 = w6_0_1 - w6_0_3;
  const T h022_0 = w6_1_0;
  const T h022_z = w6_1_1;
  const T h022_y = w6_1_2;
  const T h022_yz = w6_1_3;
  const T w7_0_0 = F[35] + F[36];
  const T w7_0_1 = F[35] - F[36];
  const T h030_0 = w7_0_0;
  const T h030_y = w7_0_1;
  const T w8_0_0 = F[1] + F[2];
  const T w8_0_1 = F[1] - F[2];
  const T h100_0 = w8_0_0;
  const T h100_x = w8_0_1;
  const T w9_0_0 = F[7] + F[13];
  const T w9_0_1 = F[7] - F[13];
  const T w9_0_2 = F[9] + F[12];
  const T w9_0_3 = F[9] - F[12];
  const T w9_0_4 = F[11] + F[10];
  const T w9_0_5 = F[11] - F[10];
  const T w9_0_6 = F[14] + F[8];
  const T w9_0_7 = F[14] - F[8];
  const T w9_1_0 = w9_0_0 + w9_0_4;
  const T w9_1_1 = w9_0_0 - w9_0_4;
  const T w9_1_2 = w9_0_1 + w9_0_5;
  const T w9_1_3 = w9_0_1 - w9_0_5;
  const T w9_1_4 = w9_0_2 + w9_0_6;
  const T w9_1_5 = w9_0_2 - w9_0_6;
  const T w9_1_6 = w9_0_3 + w9_0_7;
  const T w9_1_7 = w9_0_3 - w9_0_7;
  const T w9_2_0 = w9_1_0 + w9_1_4;
  const T w9_2_1 = w9_1_0 - w9_1_4;
  const T w9_2_2 = w9_1_1 + w9_1_5;
  const T w9_2_3 = w9_1_1 - w9_1_5;
  const T w9_2_4 = w9_1_2 + w9_1_6;
  const T w9_2_5 = w9_1_2 - w9_1_6;
  const T w9_2_6 = w9_1_3 + w9_1_7;
  const T w9_2_7 = w9_1_3 - w9_1_7;
  const T h111_0 = w9_2_0;
  const T h111_z = w9_2_1;
  const T h111_y = w9_2_2;
  const T h111_yz = w9_2_3;
  const T h111_x = w9_2_4;
  const T h111_xz = w9_2_5;
  const T h111_xy = w9_2_6;
  const T h111_xyz = w9_2_7;
  const T w10_0_0 = F[15] + F[16];
  const T w10_0_1 = F[15] - F[16];
  const T h200_0 = w10_0_0;
  const T h200_x = w10_0_1;
  const T w11_0_0 = F[25] + F[28];
  const T w11_0_1 = F[25] - F[28];
  const T w11_0_2 = F[27] + F[26];
  const T w11_0_3 = F[27] - F[26];
  const T w11_1_0 = w11_0_0 + w11_0_2;
  const T w11_1_1 = w11_0_0 - w11_0_2;
  const T w11_1_2 = w11_0_1 + w11_0_3;
  const T w11_1_3 = w11_0_1 - w11_0_3;
  const T h202_0 = w11_1_0;
  const T h202_z = w11_1_1;
  const T h202_x = w11_1_2;
  const T h202_xz = w11_1_3;
  const T w12_0_0 = F[21] + F[24];
  const T w12_0_1 = F[21] - F[24];
  const T w12_0_2 = F[23] + F[22];
  const T w12_0_3 = F[23] - F[22];
  const T w12_1_0 = w12_0_0 + w12_0_2;
  const T w12_1_1 = w12_0_0 - w12_0_2;
  const T w12_1_2 = w12_0_1 + w12_0_3;
  const T w12_1_3 = w12_0_1 - w12_0_3;
  const T h220_0 = w12_1_0;
  const T h220_y = w12_1_1;
  const T h220_x = w12_1_2;
  const T h220_xy = w12_1_3;
  const T w13_0_0 = F[33] + F[34];
  const T w13_0_1 = F[33] - F[34];
  const T h300_0 = w13_0_0;
  const T h300_x = w13_0_1;
  const T M000_0 = (((h000_0 + h010_0 + h100_0 + h220_0) + (h001_0 + h020_0 + h111_0 + h300_0)) + ((h002_0 + h022_0 + h200_0) + (h003_0 + h030_0 + h202_0)));
  const T M010_0 = ((fma(T(3), h030_y, fma(T(2), h020_y, h010_y))) + (fma(T(2), h220_y, fma(T(2), h022_y, h111_y))));
  const T M100_0 = ((fma(T(2), h220_x, fma(T(2), h200_x, h100_x))) + (fma(T(3), h300_x, fma(T(2), h202_x, h111_x))));
  const T M002_0 = ((fma(T(4), h022_0, fma(T(4), h002_0, h001_0))) + (fma(T(4), h202_0, fma(T(9), h003_0, h111_0))));
  const T M020_0 = ((fma(T(9), h030_0, fma(T(4), h020_0, h010_0))) + (fma(T(4), h220_0, fma(T(4), h022_0, h111_0))));
  const T M110_0 = fma(T(4), h220_xy, h111_xy);
  const T M200_0 = ((fma(T(4), h220_0, fma(T(4), h200_0, h100_0))) + (fma(T(9), h300_0, fma(T(4), h202_0, h111_0))));
  const T M010_1 = ((fma(T(16), h220_y, fma(T(27), h030_y, fma(T(8), h020_y, h010_y)))) + (fma(T(3), h111_y, mul_rn(T(16), h022_y))));
  const T M100_1 = ((fma(T(27), h300_x, fma(T(16), h202_x, fma(T(3), h111_x, h100_x)))) + (fma(T(16), h220_x, mul_rn(T(8), h200_x))));
  s[0] = M000_0;
  s[1] = M100_0;
  s[2] = M010_0;
  s[3] = M200_0;
  s[4] = M020_0;
  s[5] = M002_0;
  s[6] = M110_0;
  s[7] = M100_1;
  s[8] = M010_1;
}

// rho = sum f, j = sum f xi, e2f = sum f |xi|^2 (Sec. 3, macroscopic step).
template <class T, class A>
__device__ __forceinline__ void f_moments(const A& f, T& rho, T& jx, T& jy, T& jz,
                                          T& e2f) {
  const T ps1 = f[1] + f[2], pd1 = f[1] - f[2];
  const T ps3 = f[3] + f[4], pd3 = f[3] - f[4];
  const T ps5 = f[5] + f[6], pd5 = f[5] - f[6];
  const T ps7 = f[7] + f[8], pd7 = f[7] - f[8];
  const T ps9 = f[9] + f[10], pd9 = f[9] - f[10];
  const T ps11 = f[11] + f[12], pd11 = f[11] - f[12];
  const T ps13 = f[13] + f[14], pd13 = f[13] - f[14];
  const T ps15 = f[15] + f[16], pd15 = f[15] - f[16];
  const T ps17 = f[17] + f[18], pd17 = f[17] - f[18];
  const T ps19 = f[19] + f[20], pd19 = f[19] - f[20];
  const T ps21 = f[21] + f[22], pd21 = f[21] - f[22];
  const T ps23 = f[23] + f[24], pd23 = f[23] - f[24];
  const T ps25 = f[25] + f[26], pd25 = f[25] - f[26];
  const T ps27 = f[27] + f[28], pd27 = f[27] - f[28];
  const T ps29 = f[29] + f[30], pd29 = f[29] - f[30];
  const T ps31 = f[31] + f[32], pd31 = f[31] - f[32];
  const T ps33 = f[33] + f[34], pd33 = f[33] - f[34];
  const T ps35 = f[35] + f[36], pd35 = f[35] - f[36];
  const T ps37 = f[37] + f[38], pd37 = f[37] - f[38];
  rho = f[0] + (((((ps1 + ps3) + ps5) + (ps7 + ps9)) + (((ps11 + ps13) + ps15) + (ps17 + ps19))) + ((((ps21 + ps23) + ps25) + (ps27 + ps29)) + ((ps31 + ps33) + (ps35 + ps37))));
  jx = (((fma(T(2), pd25, pd1 - pd13)) + (fma(T(2), pd27, fma(T(2), pd15, pd7)))) + ((fma(T(3), pd33, fma(T(2), pd21, pd9))) + (fma(T(2), pd23, pd11))));
  jy = (((fma(T(2), pd29, pd3 - pd11)) + (fma(T(2), pd31, fma(T(2), pd17, pd7)))) + ((fma(T(3), pd35, fma(T(2), pd21, pd9))) + (fma(T(-2), pd23, pd13))));
  jz = (((fma(T(2), pd29, pd5 - pd9)) + (fma(T(-2), pd31, fma(T(2), pd19, pd7)))) + ((fma(T(3), pd37, fma(T(2), pd25, pd11))) + (fma(T(-2), pd27, pd13))));
  const T sh1 = ((ps1 + ps3) + ps5);
  const T sh3 = ((ps7 + ps9) + (ps11 + ps13));
  const T sh4 = ((ps15 + ps17) + ps19);
  const T sh8 = (((ps21 + ps23) + ps25) + ((ps27 + ps29) + ps31));
  const T sh9 = ((ps33 + ps35) + ps37);
  e2f = ((fma(T(8), sh8, fma(T(3), sh3, sh1))) + (fma(T(9), sh9, mul_rn(T(4), sh4))));
}

// sum g (the second population's share of the total energy).
template <class T, class A>
__device__ __forceinline__ T g_sum(const A& g) {
  const T gs = ((((((g[0] + g[1]) + g[2]) + (g[3] + g[4])) + (((g[5] + g[6]) + g[7]) + (g[8] + g[9]))) + ((((g[10] + g[11]) + g[12]) + (g[13] + g[14])) + (((g[15] + g[16]) + g[17]) + (g[18] + g[19])))) + (((((g[20] + g[21]) + g[22]) + (g[23] + g[24])) + (((g[25] + g[26]) + g[27]) + (g[28] + g[29]))) + ((((g[30] + g[31]) + g[32]) + (g[33] + g[34])) + ((g[35] + g[36]) + (g[37] + g[38])))));
  return gs;
}

// exp(x) = 2^(k/256) exp(r), x = k ln2/256 + r (table-driven method of P. T. P. Tang,
// ACM TOMS 15(2), 1989, with a 256-entry table): 256/ln2, ln2/256 = head + tail.
constexpr double EXP_INV_L = 369.3299304675746;
constexpr double EXP_L_HI = 0.0027076061742263846;
constexpr double EXP_L_LO = -1.6409824502660487e-13;
// 2^(j/256), j = 0..255, each the double nearest the exact value.
__device__ __constant__ double kExp2Table[256] = {
    1.0, 1.0027112750502025, 1.0054299011128027, 1.0081558981184175,
    1.0108892860517005, 1.0136300849514894, 1.016378314910953, 1.019133996077738,
    1.0218971486541166, 1.0246677928971357, 1.0274459491187637, 1.030231637686041,
    1.0330248790212284, 1.0358256936019572, 1.0386341019613787, 1.041450124688316,
    1.0442737824274138, 1.0471050958792898, 1.0499440858006872, 1.0527907730046264,
    1.0556451783605572, 1.0585073227945128, 1.061377227289262, 1.0642549128844645,
    1.0671404006768237, 1.0700337118202419, 1.0729348675259756, 1.075843889062791,
    1.0787607977571199, 1.0816856149932152, 1.0846183622133092, 1.0875590609177697,
    1.0905077326652577, 1.0934643990728858, 1.0964290818163769, 1.099401802630222,
    1.102382583307841, 1.1053714457017412, 1.1083684117236787, 1.1113735033448175,
    1.1143867425958924, 1.1174081515673693, 1.1204377524096067, 1.12347556733302,
    1.1265216186082418, 1.129575928566288, 1.1326385195987192, 1.1357094141578055,
    1.1387886347566916, 1.1418762039695616, 1.1449721444318042, 1.148076478840179,
    1.1511892299529827, 1.154310420590216, 1.1574400736337511, 1.1605782120274988,
    1.1637248587775775, 1.1668800369524817, 1.1700437696832502, 1.1732160801636373,
    1.1763969916502812, 1.1795865274628758, 1.182784710984341, 1.1859915656609938,
    1.189207115002721, 1.1924313825831512, 1.1956643920398273, 1.1989061670743806,
    1.202156731452703, 1.2054161090051239, 1.2086843236265816, 1.2119613992768012,
    1.215247359980469, 1.2185422298274085, 1.2218460329727576, 1.2251587936371455,
    1.22848053610687, 1.2318112847340759, 1.2351510639369334, 1.2384998981998165,
    1.241857812073484, 1.245224830175258, 1.2486009771892048, 1.2519862778663162,
    1.255380757024691, 1.2587844395497165, 1.2621973503942507, 1.2656195145788063,
    1.2690509571917332, 1.2724917033894028, 1.275941778396392, 1.2794012075056693,
    1.2828700160787783, 1.2863482295460256, 1.2898358734066657, 1.2933329732290895,
    1.2968395546510096, 1.3003556433796506, 1.3038812651919358, 1.3074164459346773,
    1.3109612115247644, 1.3145155879493546, 1.318079601266064, 1.3216532776031575,
    1.3252366431597413, 1.3288297242059544, 1.3324325470831615, 1.3360451382041458,
    1.339667524053303, 1.3432997311868353, 1.3469417862329458, 1.3505937158920345,
    1.3542555469368927, 1.3579273062129011, 1.3616090206382248, 1.365300717204012,
    1.3690024229745905, 1.3727141650876684, 1.3764359707545302, 1.380167867260238,
    1.383909881963832, 1.387662042298529, 1.3914243757719262, 1.3951969099662003,
    1.3989796725383112, 1.4027726912202048, 1.4065759938190154, 1.4103896082172707,
    1.4142135623730951, 1.4180478843204152, 1.4218926021691656, 1.4257477441054942,
    1.42961333839197, 1.433489413367789, 1.4373759974489824, 1.4412731191286257,
    1.4451808069770467, 1.449099089642035, 1.4530279958490526, 1.4569675544014438,
    1.460917794180647, 1.4648787441464057, 1.4688504333369818, 1.4728328908693675,
    1.4768261459394993, 1.4808302278224719, 1.4848451658727524, 1.488870989524397,
    1.4929077282912648, 1.4969554117672355, 1.5010140696264256, 1.5050837316234065,
    1.5091644275934228, 1.5132561874526098, 1.5173590411982147, 1.5214730189088146,
    1.5255981507445384, 1.529734466947287, 1.533881997840956, 1.5380407738316568,
    1.5422108254079407, 1.5463921831410214, 1.550584877685, 1.5547889397770887,
    1.559004400237837, 1.5632312899713576, 1.567469639965553, 1.5717194812923414,
    1.5759808451078865, 1.5802537626528246, 1.5845382652524937, 1.588834384317164,
    1.593142151342267, 1.597461597908627, 1.6017927556826934, 1.606135656416771,
    1.6104903319492543, 1.6148568142048607, 1.6192351351948637, 1.6236253270173289,
    1.6280274218573478, 1.632441451987275, 1.6368674497669644, 1.6413054476440063,
    1.645755478153965, 1.6502175739206177, 1.6546917676561943, 1.6591780921616162,
    1.6636765803267364, 1.6681872651305825, 1.6727101796415966, 1.6772453570178785,
    1.681792830507429, 1.6863526334483934, 1.6909247992693053, 1.6955093614893326,
    1.7001063537185235, 1.7047158096580513, 1.709337763100463, 1.713972247929926,
    1.718619298122478, 1.723278947746274, 1.7279512309618377, 1.732636182022311,
    1.7373338352737062, 1.7420442251551564, 1.746767386199169, 1.7515033530318782,
    1.7562521603732995, 1.761013843037584, 1.7657884359332727, 1.7705759740635547,
    1.7753764925265212, 1.7801900265154245, 1.785016611318935, 1.789856282321401,
    1.7947090750031072, 1.7995750249405351, 1.804454167806624, 1.809346539371032,
    1.8142521755003989, 1.8191711121586085, 1.8241033854070534, 1.8290490314048973,
    1.8340080864093424, 1.8389805867758937, 1.843966568958626, 1.8489660695104508,
    1.8539791250833855, 1.8590057724288205, 1.864046048397789, 1.8690999899412386,
    1.8741676341103, 1.8792490180565602, 1.8843441790323345, 1.8894531543909392,
    1.8945759815869656, 1.8997126981765553, 1.9048633418176741, 1.9100279502703899,
    1.9152065613971474, 1.9203992131630474, 1.925605943636125, 1.930826790987627,
    1.9360617934922943, 1.9413109895286405, 1.9465744175792332, 1.9518521162309783,
    1.9571441241754002, 1.9624504802089273, 1.9677712232331759, 1.9731063922552343,
    1.978456026387951, 1.9838201648502194, 1.9891988469672663, 1.9945921121709402,
};

}  // namespace gen
}  // namespace lbm39
