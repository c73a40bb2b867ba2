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
