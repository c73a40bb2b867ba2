// FP64 throughput probe (measurement helper; see include/ocp_probe.h).
//
// Each thread runs 8 independent dependency chains of one FP64 operation kind.  The operands
// derive from kernel parameters (1.0 and a small increment), unknown to the compiler, so no
// chain can be folded; the library is built without automatic FMA contraction, so an add stays
// a DADD and a multiply a DMUL.  The FMA comes in two forms: with its multiplier in a register
// (computed at run time) and with its multiplier read directly from the parameters (the
// constant bank), which the pipe issues at different rates.  Eight chains per thread and a few warps per scheduler give the FP64
// pipe more independent work than its latency needs, so the launch measures its issue rate.
#include <cuda_runtime.h>

#include <cstring>

#include "model_base.cuh"
#include "ocp_internal.h"
#include "ocp_probe.h"
#include "exp_table.cuh"
#include "sincos_table.cuh"

namespace {

constexpr int kChains = 8;

template <int OP>
__global__ void k_probe_fp64(double* out, int iters, double one, double eps) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double a[kChains], b[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) {
    a[k] = (double)(k + 1) * eps + (double)threadIdx.x;
    b[k] = fma(eps, (double)k, one);   // about 1, computed at run time: held in a register
  }
#pragma unroll 4
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      if (OP == 0) a[k] = fma(a[k], b[k], b[k]);       // every operand in a register
      else if (OP == 1) a[k] = a[k] + b[k];
      else if (OP == 2) a[k] = a[k] * b[k];
      else if (OP == 3) a[k] = fma(a[k], one, eps);    // multiplier a kernel parameter
      else a[k] = fma(a[k], b[k], eps);                // addend a kernel parameter, multiplier a register
    }
  }
  double s = a[0];
#pragma unroll
  for (int k = 1; k < kChains; ++k) s = s + a[k];
  out[i] = s;
}

__global__ void k_probe_recip(const double* d, double* out, int64_t n, double one) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = ocpg::recip(one, d[i]);
}

// The reduced-argument sincos (sincos_red) and the library's on the same arguments.
__global__ void k_probe_sincos(const double* x, double* s, double* c, double* sl, double* cl, int64_t n,
                               const __grid_constant__ ocpg::ModelConst K) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double a, b;
    ocpg::sincos_red(K, x[i], a, b);
    s[i] = a;
    c[i] = b;
    sincos(x[i], &a, &b);
    sl[i] = a;
    cl[i] = b;
  }
}

// The table-driven sincos (sincos_tab) and the library's on the same arguments.
__global__ void k_probe_sincos_tab(const double* x, double* s, double* c, double* sl, double* cl, int64_t n,
                                   const __grid_constant__ ocpg::ModelConst K) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double a, b;
    ocpg::sincos_tab(K, x[i], a, b);
    s[i] = a;
    c[i] = b;
    sincos(x[i], &a, &b);
    sl[i] = a;
    cl[i] = b;
  }
}

// The table-driven exponential (exp_tab) and the library's on the same arguments.
__global__ void k_probe_exp(const double* x, double* e, double* el, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    e[i] = ocpg::exp_tab(x[i], 1.0, -0.0);
    el[i] = exp(x[i]);
  }
}

}  // namespace

extern "C" ocp_status ocp_probe_exp_table(const double* x, double* e, double* e_lib, int64_t n, void* stream) {
  OCP_RANGE();
  const double* p[3] = {x, e, e_lib};
  for (const double* q : p)
    if (!q || ((uintptr_t)q & 7u)) return ocpg::set_err(nullptr, OCP_EINVAL, "ocp_probe_exp_table: bad pointer");
  if (n < 0) return ocpg::set_err(nullptr, OCP_EINVAL, "ocp_probe_exp_table: n < 0");
  if (n == 0) return OCP_OK;
  const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_probe_exp<<<grid, 256, 0, (cudaStream_t)stream>>>(x, e, e_lib, n);
  return ocpg::cuda_err(nullptr, cudaGetLastError(), "ocp_probe_exp_table launch");
}

extern "C" ocp_status ocp_probe_sincos_table(const double* x, double* s, double* c, double* s_lib, double* c_lib,
                                             int64_t n, void* stream) {
  OCP_RANGE();
  const double* p[5] = {x, s, c, s_lib, c_lib};
  for (const double* q : p)
    if (!q || ((uintptr_t)q & 7u)) return ocpg::set_err(nullptr, OCP_EINVAL, "ocp_probe_sincos_table: bad pointer");
  if (n < 0) return ocpg::set_err(nullptr, OCP_EINVAL, "ocp_probe_sincos_table: n < 0");
  if (n == 0) return OCP_OK;
  ocpg::ModelConst K;
  memset(&K, 0, sizeof(K));
  K.one = 1.0;
  K.mz = -0.0;
  const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_probe_sincos_tab<<<grid, 256, 0, (cudaStream_t)stream>>>(x, s, c, s_lib, c_lib, n, K);
  return ocpg::cuda_err(nullptr, cudaGetLastError(), "ocp_probe_sincos_table launch");
}

extern "C" ocp_status ocp_probe_sincos(const double* x, double* s, double* c, double* s_lib, double* c_lib, int64_t n,
                                       void* stream) {
  OCP_RANGE();
  const double* p[5] = {x, s, c, s_lib, c_lib};
  for (const double* q : p)
    if (!q || ((uintptr_t)q & 7u)) return ocpg::set_err(nullptr, OCP_EINVAL, "ocp_probe_sincos: bad pointer");
  if (n < 0) return ocpg::set_err(nullptr, OCP_EINVAL, "ocp_probe_sincos: n < 0");
  if (n == 0) return OCP_OK;
  ocpg::ModelConst K;
  memset(&K, 0, sizeof(K));
  K.one = 1.0;
  K.mz = -0.0;
  const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_probe_sincos<<<grid, 256, 0, (cudaStream_t)stream>>>(x, s, c, s_lib, c_lib, n, K);
  return ocpg::cuda_err(nullptr, cudaGetLastError(), "ocp_probe_sincos launch");
}

extern "C" ocp_status ocp_probe_recip(const double* d, double* out, int64_t n, void* stream) {
  OCP_RANGE();
  if (!d || !out || n < 0 || ((uintptr_t)d & 7u) || ((uintptr_t)out & 7u))
    return ocpg::set_err(nullptr, OCP_EINVAL, "ocp_probe_recip: bad arguments");
  if (n == 0) return OCP_OK;
  const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_probe_recip<<<grid, 256, 0, (cudaStream_t)stream>>>(d, out, n, 1.0);
  return ocpg::cuda_err(nullptr, cudaGetLastError(), "ocp_probe_recip launch");
}

extern "C" ocp_status ocp_probe_fp64(int op, int blocks, int threads, int iters, double* out, void* stream) {
  OCP_RANGE();
  if (op < 0 || op > 4) return ocpg::set_err(nullptr, OCP_EINVAL, "ocp_probe_fp64: op must be 0 to 4");
  if (blocks < 1 || blocks > (1 << 20) || threads < 32 || threads > 1024 || (threads & 31) || iters < 1 ||
      iters > (1 << 24))
    return ocpg::set_err(nullptr, OCP_EINVAL, "ocp_probe_fp64: blocks, threads or iters out of range");
  if (!out || ((uintptr_t)out & 7u)) return ocpg::set_err(nullptr, OCP_EINVAL, "ocp_probe_fp64: bad out pointer");
  cudaStream_t s = (cudaStream_t)stream;
  const double one = 1.0, eps = 1.0e-9;
  if (op == 0) k_probe_fp64<0><<<blocks, threads, 0, s>>>(out, iters, one, eps);
  else if (op == 1) k_probe_fp64<1><<<blocks, threads, 0, s>>>(out, iters, one, eps);
  else if (op == 2) k_probe_fp64<2><<<blocks, threads, 0, s>>>(out, iters, one, eps);
  else if (op == 3) k_probe_fp64<3><<<blocks, threads, 0, s>>>(out, iters, one, eps);
  else k_probe_fp64<4><<<blocks, threads, 0, s>>>(out, iters, one, eps);
  return ocpg::cuda_err(nullptr, cudaGetLastError(), "ocp_probe_fp64 launch");
}
