// expd.cuh -- FP64 exponential for the equilibrium evaluations.
//
// Table-driven method of P. T. P. Tang ("Table-driven implementation of the
// exponential function in IEEE floating-point arithmetic", ACM TOMS 15(2),
// 1989) with a 256-entry table: x = (256 m + j) ln2/256 + r, |r| <= ln2/512,
// exp(x) = 2^m * 2^(j/256) * exp(r), exp(r) - 1 from its degree-4 Taylor
// polynomial (truncation below 4e-17 relative).  Nine FP64 operations; the
// scaling by 2^m is an integer add to the exponent field.  The table
// 2^(j/256) and the split of ln2/256 come from gen_d3q39.py (exact decimal
// arithmetic).  exp_tang_core is valid for |x| < 512; callers route other
// arguments (and infinities, NaN) to CUDA's exp.
#pragma once
#include "d3q39_gen.cuh"

namespace lbm39 {

// Per-block copy of the table in shared memory; every kernel that evaluates
// equilibria first runs load_exp_table() with the whole block.
__device__ __forceinline__ double* exp_table() {
  __shared__ double t[256];
  return t;
}

__device__ __forceinline__ void load_exp_table() {
  double* t = exp_table();
  for (int j = threadIdx.x; j < 256; j += blockDim.x) t[j] = gen::kExp2Table[j];
  __syncthreads();
}

// 1 if |x| >= 512, x infinite or NaN.
__device__ __forceinline__ int exp_out_of_range(double x) {
  return (__double2hiint(x) & 0x7ff00000) >= ((1023 + 9) << 20);
}

__device__ __forceinline__ double exp_tang_core(double x) {
  const double shifter = 6755399441055744.0;  // 1.5 * 2^52: rounds to an integer in the low word
  const double t = fma(x, gen::EXP_INV_L, shifter);
  const int k = __double2loint(t);
  const double kd = t - shifter;
  double r = fma(kd, -gen::EXP_L_HI, x);
  r = fma(kd, -gen::EXP_L_LO, r);
  double q = fma(r, 1.0 / 24.0, 1.0 / 6.0);
  q = fma(q, r, 0.5);
  q = fma(q, r, 1.0);
  const double T = exp_table()[k & 255];
  const double y = fma(T * r, q, T);
  const int scale = (int)((unsigned)(k >> 8) << 20);  // 2^m in the exponent field
  return __hiloint2double(__double2hiint(y) + scale, __double2loint(y));
}

__device__ __forceinline__ double exp_tang(double x) {
  return exp_out_of_range(x) ? exp(x) : exp_tang_core(x);
}

}  // namespace lbm39
