// Path inequalities (paper Sec. 3: c(X_i, U_i) <= 0 at every node with a control), in the
// quadratic-plus-linear family
//     c_p(z) = sum_v [ a_{p,v} (z_v - b_{p,v})^2 + l_{p,v} z_v ] - r_p ,
// rows nb + nx N + p nun + i after the defect rows.  Their derivatives are node-local:
//     dc_p/dz_v = 2 a_{p,v} (z_v - b_{p,v}) + l_{p,v},   d2 c_p / dz_v^2 = 2 a_{p,v}.
// This kernel runs after the model's kernel of the same call on the same stream: it writes the
// path rows of c, J and J v and adds the path terms to the node's Hessian diagonal, to J^T w and
// to H v (each node's entries belong to one thread, so the additions are race-free and in a
// fixed order).  One thread per node.
#include <algorithm>
#include <cstring>

#include "ocp_internal.h"

namespace ocpg {

struct PathArgs {
  const double* __restrict__ x;
  const double* __restrict__ y;
  const double* __restrict__ vn;
  const double* __restrict__ vm;
  double *c, *jv, *hv, *ojv, *ojtv, *ohv;
  const int32_t* poff;   // terms of row p: poff[p] .. poff[p+1]-1
  const int32_t* pv;     // variable (local index) of each term
  const double* pcoef;   // a, b, l of each term (3 per term), then r (npath)
  const int64_t* jpbase; // first J slot of each path row block
  int64_t N, nun, B, E, uoff, prow0, hbase_u;
  int nx, nu, npath, nterms, hx, hu;
  int16_t hdiag[256];    // position of (v, v) in the node's X or U block (-1: none)
};

__device__ __forceinline__ int64_t path_col(const PathArgs& a, int64_t i, int v) {
  return v < a.nx ? (int64_t)a.nx * i + v : a.uoff + (int64_t)a.nu * i + (v - a.nx);
}

template <bool WC, bool WJ, bool WH, bool WJV, bool WJTV, bool WHV>
__global__ void __launch_bounds__(256) k_path(const __grid_constant__ PathArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const double* pr = a.pcoef + 3 * (int64_t)a.nterms;
  for (int64_t i = a.B + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.E; i += stride) {
    for (int p = 0; p < a.npath; ++p) {
      const int64_t row = a.prow0 + (int64_t)p * a.nun + i;
      const int t0 = __ldg(a.poff + p), t1 = __ldg(a.poff + p + 1);
      const double yp = (WH || WHV) ? __ldg(a.y + row) : 0.0;
      const double wp = WJTV ? __ldg(a.vm + row) : 0.0;
      double cv = 0.0, jvv = 0.0;
      for (int t = t0; t < t1; ++t) {
        const int v = __ldg(a.pv + t);
        const double av = __ldg(a.pcoef + 3 * t), bv = __ldg(a.pcoef + 3 * t + 1), lv = __ldg(a.pcoef + 3 * t + 2);
        const int64_t col = path_col(a, i, v);
        const double z = __ldg(a.x + col);
        const double d = z - bv;
        if (WC) cv = cv + (av * d * d + lv * z);
        const double dv = 2.0 * av * d + lv;   // dc_p / dz_v
        if (WJ) a.jv[a.jpbase[p] + i * (t1 - t0) + (t - t0)] = dv;
        if (WJV) jvv = jvv + dv * __ldg(a.vn + col);
        if (WJTV) a.ojtv[col] = a.ojtv[col] + wp * dv;
        if (av != 0.0) {  // the squared term's diagonal
          const double h2 = 2.0 * av * yp;
          if (WH) {
            const int e = a.hdiag[v];
            const int64_t slot = v < a.nx ? (int64_t)a.hx * i + e : a.hbase_u + (int64_t)a.hu * i + e;
            a.hv[slot] = a.hv[slot] + h2;
          }
          if (WHV) a.ohv[col] = a.ohv[col] + h2 * __ldg(a.vn + col);
        }
      }
      if (WC) a.c[row] = cv - __ldg(pr + p);
      if (WJV) a.ojv[row] = jvv;
    }
  }
}

static ocp_status path_fill(const ocp* h, PathArgs& a, int64_t B, int64_t E) {
  const Pattern& P = h->pat;
  memset(&a, 0, sizeof(a));
  if (P.nz > 256) return OCP_EDIM;
  a.poff = h->d_poff; a.pv = h->d_pv; a.pcoef = h->d_pcoef; a.jpbase = h->d_pbase;
  a.N = h->N; a.nun = P.nun;
  a.B = B; a.E = std::min(E, P.nun);
  a.uoff = (int64_t)h->nx * (h->N + 1);
  a.prow0 = P.nb + (int64_t)h->nx * h->N;
  a.hbase_u = P.hbase_u;
  a.nx = h->nx; a.nu = h->nu; a.npath = P.npath; a.hx = P.hx; a.hu = P.hu;
  for (int p = 0; p < P.npath; ++p) a.nterms += (int)P.psupp[p].size();
  for (int v = 0; v < P.nz; ++v) a.hdiag[v] = (int16_t)P.hdiag[v];
  return OCP_OK;
}

template <bool WC, bool WJ, bool WH, bool WJV, bool WJTV, bool WHV>
static cudaError_t path_go(const ocp* h, const PathArgs& a, cudaStream_t s) {
  const int64_t n = a.E - a.B;
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)h->num_sms * 8);
  k_path<WC, WJ, WH, WJV, WJTV, WHV><<<(int)std::max<int64_t>(blocks, 1), 256, 0, s>>>(a);
  return cudaGetLastError();
}

ocp_status path_eval(ocp* h, unsigned out, const EvalCall& c, cudaStream_t s) {
  if (h->pat.npath == 0) return OCP_OK;
  PathArgs a;
  if (path_fill(h, a, c.B, c.E) != OCP_OK) return set_err(h, OCP_EDIM, "too many variables per node for path rows");
  a.x = c.x; a.y = c.y; a.vn = c.vn; a.vm = c.vm;
  a.c = c.c; a.jv = c.jv; a.hv = c.hv; a.ojv = c.ojv; a.ojtv = c.ojtv; a.ohv = c.ohv;
  const bool C = c.c, J = c.jv, H = c.hv, JV = c.ojv, JT = c.ojtv, HV = c.ohv;
  cudaError_t e = cudaSuccess;
  if (JV || JT || HV) {  // the fused step: every output
    e = path_go<true, true, true, true, true, true>(h, a, s);
  } else {
    if (C && J && H) e = path_go<true, true, true, false, false, false>(h, a, s);
    else if (J && H) e = path_go<false, true, true, false, false, false>(h, a, s);
    else {
      if (C && e == cudaSuccess) e = path_go<true, false, false, false, false, false>(h, a, s);
      if (J && e == cudaSuccess) e = path_go<false, true, false, false, false, false>(h, a, s);
      if (H && e == cudaSuccess) e = path_go<false, false, true, false, false, false>(h, a, s);
    }
  }
  return cuda_err(h, e, "path rows launch");
}

ocp_status path_prod(ocp* h, const ProdCall& c, cudaStream_t s) {
  if (h->pat.npath == 0) return OCP_OK;
  PathArgs a;
  const int64_t B = (c.kind == P_JTPROD) ? c.B : 0, E = (c.kind == P_JTPROD && c.E >= 0) ? c.E : h->N + 1;
  if (path_fill(h, a, B, E) != OCP_OK) return set_err(h, OCP_EDIM, "too many variables per node for path rows");
  a.x = c.x; a.y = c.y;
  cudaError_t e;
  if (c.kind == P_JPROD) { a.vn = c.v; a.ojv = c.out; e = path_go<false, false, false, true, false, false>(h, a, s); }
  else if (c.kind == P_JTPROD) { a.vm = c.v; a.ojtv = c.out; e = path_go<false, false, false, false, true, false>(h, a, s); }
  else { a.vn = c.v; a.ohv = c.out; e = path_go<false, false, false, false, false, true>(h, a, s); }
  return cuda_err(h, e, "path rows launch");
}

// Device tables of the path rows (terms, coefficients, slot bases); called after every
// pattern rebuild.
ocp_status path_upload(ocp* h) {
  cudaFree(h->d_poff); cudaFree(h->d_pv); cudaFree(h->d_pcoef); cudaFree(h->d_pbase);
  h->d_poff = nullptr; h->d_pv = nullptr; h->d_pcoef = nullptr; h->d_pbase = nullptr;
  const Pattern& P = h->pat;
  std::vector<int32_t> poff(1, 0), pv;
  std::vector<double> coef;
  for (int p = 0; p < P.npath; ++p) {
    for (int v : P.psupp[p]) {
      pv.push_back(v);
      coef.push_back(h->path_a[p * P.nz + v]);
      coef.push_back(h->path_b[p * P.nz + v]);
      coef.push_back(h->path_l[p * P.nz + v]);
    }
    poff.push_back((int32_t)pv.size());
  }
  for (int p = 0; p < P.npath; ++p) coef.push_back(h->path_r[p]);
  std::vector<int64_t> base(P.jpbase);
  base.insert(base.end(), P.kpbase.begin(), P.kpbase.end());
  if (pv.empty()) pv.push_back(0);
  if (coef.empty()) coef.push_back(0.0);
  cudaError_t e;
  if ((e = ocpg::dev_malloc(&h->d_poff, poff.size() * 4)) != cudaSuccess ||
      (e = ocpg::dev_malloc(&h->d_pv, pv.size() * 4)) != cudaSuccess ||
      (e = ocpg::dev_malloc(&h->d_pcoef, coef.size() * 8)) != cudaSuccess ||
      (e = ocpg::dev_malloc(&h->d_pbase, base.size() * 8)) != cudaSuccess)
    return cuda_err(h, e, "cudaMalloc(path tables)");
  if ((e = ocpg::dev_upload(h->d_poff, poff.data(), poff.size() * 4)) != cudaSuccess ||
      (e = ocpg::dev_upload(h->d_pv, pv.data(), pv.size() * 4)) != cudaSuccess ||
      (e = ocpg::dev_upload(h->d_pcoef, coef.data(), coef.size() * 8)) != cudaSuccess ||
      (e = ocpg::dev_upload(h->d_pbase, base.data(), base.size() * 8)) != cudaSuccess)
    return cuda_err(h, e, "cudaMemcpy(path tables)");
  return OCP_OK;
}

}  // namespace ocpg
