// Common part of the device models of the dynamics x' = f(x, u) (paper Sec. 3) with hand-derived derivatives.
//
// Every model describes, at compile time, the sparsity template of one node:
//   - for each state component k, the Jacobian row template of the defect c_{k,j}: the
//     X-local variables XV(k, .) (sorted, always including k itself for the identity term of
//     the trapezoidal defect) and the U-local variables UV(k, .) whose derivative
//     df_k/dz_v is not identically zero; JZ(k, e) marks entries that are the identity term
//     alone (df_k/dz_v identically 0);
//   - the pairs (HA(e) >= HB(e)) of local variables with a Hessian of some f_k not
//     identically zero, and HK(k): whether f_k has a Hessian at all.
// The host pattern compiler reads these tables; the kernels place values by them.
//
// At one node z = (x, u) a model returns, with hh = h/2:
//   pa[k] = x_k + hh f_k(z),  pb[k] = x_k - hh f_k(z)   (defect (k,j) = pb(j+1) - pa(j))
//   mjx[k][e] = -hh df_k/dx_{XV(k,e)}(z)   (identity excluded),  mju[k][e] = -hh df_k/du_{UV(k,e)}(z)
//   hd[e] = -hh sum_k ybar_k d2 f_k/dz_{HA(e)} dz_{HB(e)}(z)  (+ cqd[a] on a diagonal entry),
// where cqd is the diagonal of sigma * w_j * Hess f0 at this node.  A Jacobian value is then
// mjx - 1 (left node, identity), mjx + 1 (right node, identity) or the bare mjx / mju.
//
// The library is compiled with automatic FMA contraction off: every FMA below is explicit,
// so the FP64 operation count is what the source says (GB300 executes FP64 at 2 FMA per
// clock per SM, which bounds these kernels) and every kernel variant rounds identically.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ocpg {

// Kernel-side model constants (filled by the host from the handle's parameters).
struct ModelConst {
  double hh;       // h / 2
  double mhh;      // -h / 2
  double one;      // 1.0 and -0.0, passed at run time (see fadd / fmul below)
  double mz;
  double c[16];    // model-specific precomputed constants (see each model)
};

// GB300's FP64 pipe sustains FMAs at its full rate but separate adds and multiplies about 18%
// slower (measured), so sums, differences and products are issued as FMAs against the run-time
// constants 1 and -0: a + b = fma(a, 1, b), a - b = fma(-b, 1, a), a * b = fma(a, b, -0).
// These round exactly like the plain operations (signed zeros included); the constants come
// from kernel parameters so that the compiler cannot fold the FMAs back.
__device__ __forceinline__ double fadd(const ModelConst& K, double a, double b) { return fma(a, K.one, b); }
__device__ __forceinline__ double fsub(const ModelConst& K, double a, double b) { return fma(-b, K.one, a); }
__device__ __forceinline__ double fmul(const ModelConst& K, double a, double b) { return fma(a, b, K.mz); }

// Operand sources matter as well (measured with the library's FP64 throughput probe, all
// operands independent): an FMA whose multiplier is a register issues at the pipe's full rate,
// 2 per clock per SM, but at about 5/6 of it when the multiplier is read from the constant bank
// (a kernel parameter used directly), and DADD and DMUL run at 5/6 too.  Taking the constants
// through shared memory puts them in registers, but in these kernels the extra registers cost
// more occupancy than the faster FMAs gain (measured on the fused step: whole argument block
// 110.6-127.9 us, model constants only 109.3-112.9 us, the constant 1 alone 108.7 us, against
// 106.0 us from the constant bank), so the kernels read their constants from the parameters.
// 1 / d by Newton-Raphson iteration for the reciprocal, r <- r + r (1 - d r) (each step squares
// the relative error), started from the hardware's approximate reciprocal (PTX
// rcp.approx.ftz.f64, relative error below 2^-22, computed by the special-function unit, not the
// FP64 pipe): two steps reach FP64 accuracy, within an ulp of the correctly rounded 1 / d, with
// four FMAs, where the IEEE division costs more FP64 instructions.  For finite, normal d: the
// models' denominators are bounded away from zero (a subnormal d is flushed to zero, d = 0 gives
// NaN instead of infinity).
// (`one` is the run-time constant 1.)
__device__ __forceinline__ double recip(double one, double d) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
  double e = fma(-d, r, one);
  r = fma(r, e, r);
  e = fma(-d, r, one);
  return fma(r, e, r);
}

// sin x and cos x together, without the library routine's branches (CUDA's sincos executes about
// 19 FP64 instructions and leaves about five predicated-off ones in the pipe, measured as the
// excess of warp-level FP64 instructions x 32 over the thread-level count; this one executes
// 24 with no predicated ones: the same pipe slots, fewer branches and other instructions, and
// on the cart-pole J^T w 151.7 -> 145.5 us, J + H 180.2 -> 179.3 us at N = 1e6).  Method (Cody and Waite, "Software Manual for the Elementary
// Functions", 1980, with the reduction constant split in three): |x| = k pi/2 + r with k the
// integer nearest 2|x|/pi (rounded by adding 1.5 2^52, whose low mantissa bits then hold k mod
// 2^32) and r = ((|x| - k P1) - k P2) - k P3, P1 + P2 + P3 = pi/2 (each the double nearest the
// remainder; the first step is exact for |x| <= 1e5, both terms being multiples of 2^-52);
// then the Taylor series of sin r through r^17 and of cos r through r^16, whose truncation
// errors on |r| <= pi/4 are below 2e-19 and 3e-18 relative, by Horner's rule in z = r^2 with the
// coefficients +-1/n! rounded to double; the quadrant k mod 4 swaps and negates (sign bits
// only).  The reduction runs on |x| and sin takes the sign of x (sin is odd, cos even), which
// keeps sin(-0) = -0.  Within about two ulps of the correctly rounded values (checked against the library
// by ocp_probe_sincos).  A warp whose active lanes are not all finite with |x| <= 1e5 takes the
// library routine (the branch is uniform: no predicated instructions on the common path).
__device__ __forceinline__ void sincos_red(const ModelConst& K, double x, double& s, double& c) {
  if (__all_sync(__activemask(), fabs(x) <= 1.0e5)) {
    const double ax = fabs(x);
    const double t = fma(ax, 0x1.45f306dc9c883p-1, 0x1.8p52);  // 2/pi
    const double k = fsub(K, t, 0x1.8p52);
    double r = fma(-k, 0x1.921fb54442d18p+0, ax);              // P1
    r = fma(-k, 0x1.1a62633145c07p-54, r);                     // P2
    r = fma(-k, -0x1.f1976b7ed8fbcp-110, r);                   // P3
    const double z = fmul(K, r, r);
    double ps = fma(z, 0x1.952c77030ad4ap-49, -0x1.ae7f3e733b81fp-41);   // 1/17!, -1/15!
    ps = fma(z, ps, 0x1.6124613a86d09p-33);                              // 1/13!
    ps = fma(z, ps, -0x1.ae64567f544e4p-26);                             // -1/11!
    ps = fma(z, ps, 0x1.71de3a556c734p-19);                              // 1/9!
    ps = fma(z, ps, -0x1.a01a01a01a01ap-13);                             // -1/7!
    ps = fma(z, ps, 0x1.1111111111111p-7);                               // 1/5!
    ps = fma(z, ps, -0x1.5555555555555p-3);                              // -1/3!
    const double sr = fma(fmul(K, r, z), ps, r);
    double pc = fma(z, 0x1.ae7f3e733b81fp-45, -0x1.93974a8c07c9dp-37);   // 1/16!, -1/14!
    pc = fma(z, pc, 0x1.1eed8eff8d898p-29);                              // 1/12!
    pc = fma(z, pc, -0x1.27e4fb7789f5cp-22);                             // -1/10!
    pc = fma(z, pc, 0x1.a01a01a01a01ap-16);                              // 1/8!
    pc = fma(z, pc, -0x1.6c16c16c16c17p-10);                             // -1/6!
    pc = fma(z, pc, 0x1.5555555555555p-5);                               // 1/4!
    pc = fma(z, pc, -0.5);                                               // -1/2!
    const double cr = fma(z, pc, 1.0);
    const int q = __double2loint(t);                           // k mod 4 in the low bits
    const double a = (q & 1) ? cr : sr, b = (q & 1) ? sr : cr;
    // sin |x| = (sr, cr, -sr, -cr), cos |x| = (cr, -sr, -cr, sr) for k mod 4 = 0..3
    s = __hiloint2double(__double2hiint(a) ^ ((q & 2) << 30) ^ (__double2hiint(x) & (int)0x80000000),
                         __double2loint(a));
    c = __hiloint2double(__double2hiint(b) ^ (((q + 1) & 2) << 30), __double2loint(b));
  } else {
    sincos(x, &s, &c);
  }
}

// Size of a per-parameter array of model M (at least 1; M::NP = 0 has no parameters).
template <class M>
__host__ __device__ constexpr int npa() { return M::NP > 0 ? M::NP : 1; }

#define OCP_TABLE1(NAME, TYPE, N, ...)                       \
  __host__ __device__ static constexpr TYPE NAME(int k) {    \
    constexpr TYPE t[N] = __VA_ARGS__;                       \
    return t[k];                                             \
  }
#define OCP_TABLE2(NAME, TYPE, N, M, ...)                        \
  __host__ __device__ static constexpr TYPE NAME(int k, int e) { \
    constexpr TYPE t[N][M] = __VA_ARGS__;                        \
    return t[k][e];                                              \
  }

}  // namespace ocpg
