// Table-driven exponential of the Goddard rocket's drag term.
#pragma once
#include <cuda_runtime.h>

namespace ocpg {

#include "exp_table_data.h"

// exp(x) by table lookup (the table-driven method of P. T. P. Tang, "Table-driven implementation
// of the exponential function in IEEE floating-point arithmetic", ACM TOMS 15(2), 1989):
// k = 32 m + j is the integer nearest 32 x / ln 2 (rounded by adding 1.5 2^52, whose low mantissa
// bits then hold k) and r = (x - k L1) - k L2 with L1 + L2 = ln 2 / 32 (each the double nearest
// the remainder), so |r| <= ln 2 / 64; then
//   exp(x) = 2^m 2^(j/32) (1 + p(r)),  p(r) = r + r^2 (1/2 + r (1/6 + r (1/24 + r (1/120 + r/720)))),
// the omitted terms of the series below 4e-18 of the result; 2^(j/32) comes from kExp2Table (the
// doubles nearest the exact values) and 2^m is added to the exponent bits.  11 FP64 instructions;
// within one ulp of the correctly rounded value (ocp_probe_exp_table).  `one` and `mz` are the
// run-time constants 1 and -0 (the sum and the product by which the kernels issue their adds and
// multiplies as FMAs).  A warp whose active lanes are not all finite with |x| <= 700 takes the
// library routine (a uniform branch), so the scaled result stays a normal number.
__device__ __forceinline__ double exp_tab(double x, double one, double mz) {
  if (__all_sync(__activemask(), fabs(x) <= 700.0)) {
    const double t = fma(x, 0x1.71547652b82fep+5, 0x1.8p52);  // 32 / ln 2
    const double k = fma(-0x1.8p52, one, t);
    double r = fma(-k, 0x1.62e42fefa39efp-6, x);                // L1
    r = fma(-k, 0x1.abc9e3b39803fp-61, r);                      // L2
    const int ki = __double2loint(t);                           // k (|k| < 2^15)
    const double tj = __ldg(&kExp2Table[ki & 31]);
    double q = fma(r, 0x1.6c16c16c16c17p-10, 0x1.1111111111111p-7);  // 1/6!, 1/5!
    q = fma(r, q, 0x1.5555555555555p-5);                              // 1/4!
    q = fma(r, q, 0x1.5555555555555p-3);                              // 1/3!
    q = fma(r, q, 0.5);                                               // 1/2!
    const double p = fma(fma(r, r, mz), q, r);
    const double e = fma(tj, p, tj);
    return __hiloint2double(__double2hiint(e) + (ki >> 5) * (1 << 20), __double2loint(e));
  }
  return exp(x);
}

}  // namespace ocpg
