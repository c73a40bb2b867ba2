// Table-driven sine and cosine of the models with trigonometric dynamics (the cart-pole's pole
// angle, the quadrotor's three attitude angles).
#pragma once
#include "model_base.cuh"

namespace ocpg {

#include "sincos_table_data.h"

// sin x and cos x together by table lookup (the table-lookup method of P. T. P. Tang, "Table-
// lookup algorithms for elementary functions and their error analysis", ARITH 10, 1991, here
// for the pair sin, cos):  |x| = k pi/512 + r with k the integer nearest 512|x|/pi (rounded by
// adding 1.5 2^52, whose low mantissa bits then hold k) and r = ((|x| - k P1) - k P2) - k P3,
// P1 + P2 + P3 = pi/512 (each the double nearest the remainder), so |r| <= pi/1024.  With
// a = (k mod 256) pi/512 in [0, pi/2) and the quadrant q = (k div 256) mod 4,
//   sin(a + r) = sin a + (sin a (cos r - 1) + cos a sin r),
//   cos(a + r) = cos a + (cos a (cos r - 1) - sin a sin r),
// where sin a, cos a come from kSinCosTable (the doubles nearest the exact values), sin r =
// r - r^3/6 + r^5/120 and cos r - 1 = -r^2/2 + r^4/24 (the omitted terms are below 2e-19 of the
// result on |r| <= pi/1024); the quadrant then swaps and negates (sign bits only) and sin takes
// the sign of x (sin is odd, cos even), which keeps sin(-0) = -0.  15 FP64 instructions, against
// 24 for sincos_red's Taylor polynomials on |r| <= pi/4; within two ulps of the correctly
// rounded values (ocp_probe_sincos_table).  A warp whose active lanes are not all finite with
// |x| <= 1e5 takes the library routine (a uniform branch).
__device__ __forceinline__ void sincos_tab(const ModelConst& K, double x, double& s, double& c) {
  if (__all_sync(__activemask(), fabs(x) <= 1.0e5)) {
    const double ax = fabs(x);
    const double t = fma(ax, 0x1.45f306dc9c883p+7, 0x1.8p52);   // 512/pi
    const double k = fsub(K, t, 0x1.8p52);
    double r = fma(-k, 0x1.921fb54442d18p-8, ax);                // P1
    r = fma(-k, 0x1.1a62633145c07p-62, r);                       // P2
    r = fma(-k, -0x1.f1976b7ed8fbcp-118, r);                     // P3
    const int ki = __double2loint(t);                            // k mod 2^32
    const double2 sc = __ldg(&kSinCosTable[ki & 255]);           // sin a, cos a
    const double z = fmul(K, r, r);
    const double sr = fma(fmul(K, r, z), fma(z, 0x1.1111111111111p-7, -0x1.5555555555555p-3), r);  // 1/5!, -1/3!
    const double cm1 = fmul(K, z, fma(z, 0x1.5555555555555p-5, -0.5));                          // 1/4!, -1/2!
    const double sy = fma(sc.y, sr, fma(sc.x, cm1, sc.x));
    const double cy = fma(-sc.x, sr, fma(sc.y, cm1, sc.y));
    const int q = ki >> 8;
    const double a = (q & 1) ? cy : sy, b = (q & 1) ? sy : cy;
    // sin |x| = (sy, cy, -sy, -cy), cos |x| = (cy, -sy, -cy, sy) for q mod 4 = 0..3
    s = __hiloint2double(__double2hiint(a) ^ ((q & 2) << 30) ^ (__double2hiint(x) & (int)0x80000000),
                         __double2loint(a));
    c = __hiloint2double(__double2hiint(b) ^ (((q + 1) & 2) << 30), __double2loint(b));
  } else {
    sincos(x, &s, &c);
  }
}

}  // namespace ocpg
