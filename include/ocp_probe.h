/*
 * ocp_probe.h — measurement helper of the evaluator library (not part of the paper's method).
 *
 * The evaluation kernels of ocp.h are bound by the GPU's FP64 pipe, so their roofline is an
 * FP64 instruction rate.  This call runs a throughput kernel of one FP64 operation kind so that
 * a benchmark can measure that rate on the GPU it runs on, at the clocks of the same run,
 * instead of quoting a data-sheet figure.
 */
#ifndef OCP_GB300_PROBE_H
#define OCP_GB300_PROBE_H

#include <stdint.h>

#include "ocp.h"

#ifdef __cplusplus
extern "C" {
#endif

/* FP64 throughput probe.  op: 0 = fused multiply-add (DFMA) with every operand in a register,
 * 1 = add (DADD), 2 = multiply (DMUL), 3 = DFMA whose multiplier is a kernel parameter (read
 * from the constant bank), 4 = DFMA whose addend is a kernel parameter.  Launches `blocks` CTAs of `threads` threads (threads a multiple of 32, at most
 * 1024); each thread runs 8 independent dependency chains of `iters` operations of that kind,
 * so one launch executes blocks * threads * 8 * iters FP64 operations (plus 7 adds per thread
 * that combine the chains).  Each thread writes one double to `out` (device, at least
 * blocks * threads doubles; the values are meaningless).  The call
 * is asynchronous on `stream`; the caller times it (e.g. with CUDA events on that stream).
 * Errors: OCP_EINVAL for a bad op, size or pointer; OCP_ECUDA for a failed launch, with
 * ocp_last_error(NULL). */
ocp_status ocp_probe_fp64(int op, int blocks, int threads, int iters, double* out, void* stream);

/* The evaluation kernels' reciprocal 1/d (Newton-Raphson steps from the hardware's approximate
 * reciprocal) on n values: out[i] = recip(d[i]) (device arrays; asynchronous on `stream`), so
 * that a test can compare it with the IEEE division.  For finite, normal d.  Errors: OCP_EINVAL,
 * OCP_ECUDA (ocp_last_error(NULL)). */
ocp_status ocp_probe_recip(const double* d, double* out, int64_t n, void* stream);

/* The library's reduced-argument sin and cos (a three-constant Cody-Waite reduction to
 * |r| <= pi/4 and Taylor polynomials, with CUDA's routine for warps holding an argument beyond
 * 1e5 or not finite; the evaluation kernels used it before the table-driven routine below
 * replaced it) and CUDA's sincos on the same n arguments: s[i], c[i] and s_lib[i], c_lib[i]
 * (device arrays; asynchronous on `stream`), so that a test can bound the difference.  Errors:
 * OCP_EINVAL, OCP_ECUDA (ocp_last_error(NULL)). */
ocp_status ocp_probe_sincos(const double* x, double* s, double* c, double* s_lib, double* c_lib, int64_t n,
                            void* stream);

/* The same for the table-driven sin and cos of the cart-pole and quadrotor kernels (|x| = k pi/512
 * + r, sin and cos of k pi/512 from a table of the doubles nearest the exact values, short
 * polynomials in r, the library routine for warps holding an argument beyond 1e5 or not
 * finite): s[i], c[i], and CUDA's sincos in s_lib[i], c_lib[i] (device arrays; asynchronous on
 * `stream`).  Errors: OCP_EINVAL, OCP_ECUDA (ocp_last_error(NULL)). */
ocp_status ocp_probe_sincos_table(const double* x, double* s, double* c, double* s_lib, double* c_lib, int64_t n,
                                  void* stream);

/* The Goddard kernels' table-driven exponential (x = (32 m + j) ln 2/32 + r, 2^(j/32) from a table
 * of the doubles nearest the exact values, a degree-6 polynomial in r, 2^m on the exponent
 * bits; the library routine for warps holding an argument beyond 700 in magnitude or not
 * finite) and CUDA's exp on the same n arguments: e[i] and e_lib[i] (device arrays;
 * asynchronous on `stream`).  Errors: OCP_EINVAL, OCP_ECUDA (ocp_last_error(NULL)). */
ocp_status ocp_probe_exp_table(const double* x, double* e, double* e_lib, int64_t n, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* OCP_GB300_PROBE_H */
