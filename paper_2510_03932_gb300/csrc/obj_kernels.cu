// Objective-only kernels for the differentiation form (any model: the running cost is the
// diagonal quadratic f0 = sum_v q_v (z_v - ref_v)^2, so only the cost coefficients and the
// reference matter; a tracked state's ref_v(t_j) comes from the per-node table):
//   g  = s * grad F(x)                       (s a device scalar: the upstream gradient)
//   Hv = s * Hess F(x) v,  dot = grad F(x) . v   (double backward of the objective)
// with  grad F_{j,v} = 2 w_j q_v (z_v - ref_v)  and  Hess F = diag(2 w_j q_v)  (paper Sec. 5
// trapezoidal cost: w_0 = w_N = h/2, w_j = h otherwise).  One thread per node; the dot
// product is reduced per tile and the tiles are summed in order (deterministic).
#include <cstring>

#include "node_kernels.cuh"
#include "ocp_internal.h"

namespace ocpg {

constexpr int OBJ_THREADS = 256;
constexpr int OBJ_MAXV = 129;

struct ObjArgs {
  const double* __restrict__ x;
  const double* __restrict__ v;
  const double* __restrict__ s;   // device scalar
  double* out;
  double* dot;
  double* partials;
  unsigned* counter;
  int64_t N, uoff;
  int nx, nu, has_ref;
  double one, mz;   // 1.0 and -0.0 at run time: sums and products are issued as FMAs
  const double* xtrack;  // time-varying state reference, (N+1) x ntrk node-major, or null
  int ntrk;
  double gq_in[OBJ_MAXV], gq_end[OBJ_MAXV], ref[OBJ_MAXV];
  int trk[OBJ_MAXV];     // column of state v in xtrack, or -1
};

__device__ __forceinline__ int64_t var_index(const ObjArgs& a, int64_t j, int v) {
  return v < a.nx ? (int64_t)a.nx * j + v : a.uoff + (int64_t)a.nu * j + (v - a.nx);
}

// HVP = false: out = s * grad F.   HVP = true: out = s * Hess F v, dot = grad F . v
template <bool HVP>
__global__ void __launch_bounds__(OBJ_THREADS) k_obj(const __grid_constant__ ObjArgs a) {
  __shared__ double red[OBJ_THREADS];
  const double s = __ldg(a.s);
  const int nz = a.nx + a.nu;
  const int64_t nchunks = (a.N + OBJ_THREADS) / OBJ_THREADS;
  for (int64_t chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
    const int64_t j = chunk * OBJ_THREADS + threadIdx.x;
    double acc = 0.0;
    if (j <= a.N) {
      const bool endp = (j == 0) || (j == a.N);
      for (int v = 0; v < nz; ++v) {
        const int64_t idx = var_index(a, j, v);
        const double gq = endp ? a.gq_end[v] : a.gq_in[v];   // 2 w_j q_v
        const double z = __ldg(a.x + idx);
        double rv = a.ref[v];
        if (v < a.nx && a.xtrack && a.trk[v] >= 0) rv = __ldg(a.xtrack + (int64_t)a.ntrk * j + a.trk[v]);
        const double d = a.has_ref ? fma(-rv, a.one, z) : z;
        const double sg = fma(s, gq, a.mz);
        if (HVP) {
          const double vv = __ldg(a.v + idx);
          a.out[idx] = fma(sg, vv, a.mz);
          acc = fma(fma(gq, d, a.mz), vv, acc);
        } else {
          a.out[idx] = fma(sg, d, a.mz);
        }
      }
    }
    if (HVP && a.dot) {
      const double ts = tile_sum<OBJ_THREADS>(acc, red, a.one);
      if (threadIdx.x == 0) a.partials[chunk] = ts;
      __syncthreads();
    }
  }
  if (HVP && a.dot) finish_tiles<OBJ_THREADS>(a.partials, nchunks, a.counter, a.dot, 1.0, red);
}

ocp_status obj_launch(ocp* h, bool hvp, const double* x, const double* s, const double* v, double* out,
                      double* dot, cudaStream_t st) {
  const int nz = h->nx + h->nu;
  if (nz > OBJ_MAXV) return set_err(h, OCP_EDIM, "too many variables per node for the objective kernel");
  if (h->model == OCP_MODEL_GODDARD)
    return set_err(h, OCP_EMODEL, "the objective kernels cover running costs (Goddard has a terminal cost)");
  if (h->scheme != OCP_SCHEME_TRAPEZOID)
    return set_err(h, OCP_EMODEL, "the objective kernels use the trapezoidal weights");
  ObjArgs a;
  memset(&a, 0, sizeof(a));
  a.x = x; a.v = v; a.s = s; a.out = out; a.dot = dot;
  a.partials = h->d_partials; a.counter = h->d_counter;
  a.N = h->N; a.uoff = (int64_t)h->nx * (h->N + 1);
  a.nx = h->nx; a.nu = h->nu; a.has_ref = h->has_ref ? 1 : 0;
  a.one = 1.0;
  a.mz = -0.0;
  a.xtrack = h->d_xtrack;
  a.ntrk = h->ntrk;
  for (int v2 = 0; v2 < OBJ_MAXV; ++v2) a.trk[v2] = -1;
  for (int i = 0; i < h->ntrk; ++i) a.trk[h->trk_comp[i]] = i;
  for (int v2 = 0; v2 < nz; ++v2) {
    const double w = v2 < h->nx ? h->q[v2] : h->r[v2 - h->nx];
    a.gq_in[v2] = 2.0 * h->h * w;
    a.gq_end[v2] = h->h * w;
    a.ref[v2] = v2 < h->nx ? h->xref[v2] : h->uref[v2 - h->nx];
  }
  const int64_t nchunks = (h->N + OBJ_THREADS) / OBJ_THREADS;
  const int grid = occupancy_grid(h, nullptr, OBJ_THREADS, 0, nchunks);
  if (hvp) k_obj<true><<<grid, OBJ_THREADS, 0, st>>>(a);
  else k_obj<false><<<grid, OBJ_THREADS, 0, st>>>(a);
  return cuda_err(h, cudaGetLastError(), "objective kernel launch");
}

}  // namespace ocpg
