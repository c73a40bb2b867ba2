// Boundary terms on (X_0, X_N): the inequalities b(X_0, X_N) <= 0 and the boundary cost g(X_0,
// X_N) of the objective (both paper Sec. 3).
// Boundary inequalities (paper Sec. 3: b(X_0, X_N) <= 0) in the quadratic-plus-linear family
//     b_q(z) = sum_v [ a_{q,v} (z_v - b_{q,v})^2 + l_{q,v} z_v ] - r_q ,   z = (X_0, X_N),
// rows nb + nx N + npath nun + q after the path rows.  Derivatives:
//     db_q/dz_v = 2 a_{q,v} (z_v - b_{q,v}) + l_{q,v},   d2 b_q / dz_v^2 = 2 a_{q,v}.
// The rows couple the first and the last node, and there are few of them: one thread
// evaluates them all, in row order, after the model's and the path rows' kernels on the same
// stream.  It writes the rows of c, J and J v and adds the rows' terms to the Hessian
// diagonals of nodes 0 and N, to J^T w and to H v (a fixed order of additions).
#include <algorithm>
#include <cstring>

#include "ocp_internal.h"

namespace ocpg {

struct BinArgs {
  const double* __restrict__ x;
  const double* __restrict__ y;
  const double* __restrict__ vn;
  const double* __restrict__ vm;
  double *c, *jv, *hv, *ojv, *ojtv, *ohv;
  const int32_t* boff;   // terms of row q: boff[q] .. boff[q+1]-1
  const int32_t* bv;     // variable of each term (local index of z)
  const double* bcoef;   // a, b, l of each term (3 per term), then r (nbin)
  const int64_t* jbase;  // first J slot of each row
  int64_t N, brow0, xN;  // xN: column of X_{N,0}
  int nx, nbin, nterms, hx;
  int16_t hdiag[256];    // position of (k, k) in the node's X block (-1: none)
};

template <bool WC, bool WJ, bool WH, bool WJV, bool WJTV, bool WHV>
__global__ void __launch_bounds__(32) k_bin(const __grid_constant__ BinArgs a) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double* br = a.bcoef + 3 * (int64_t)a.nterms;
  for (int q = 0; q < a.nbin; ++q) {
    const int64_t row = a.brow0 + q;
    const int t0 = a.boff[q], t1 = a.boff[q + 1];
    const double yq = (WH || WHV) ? a.y[row] : 0.0;
    const double wq = WJTV ? a.vm[row] : 0.0;
    double cv = 0.0, jvv = 0.0;
    for (int t = t0; t < t1; ++t) {
      const int v = a.bv[t];
      const double av = a.bcoef[3 * t], bv = a.bcoef[3 * t + 1], lv = a.bcoef[3 * t + 2];
      const bool fin = v >= a.nx;
      const int k = fin ? v - a.nx : v;
      const int64_t col = fin ? a.xN + k : (int64_t)k;
      const double z = a.x[col];
      const double d = z - bv;
      if (WC) cv = cv + (av * d * d + lv * z);
      const double dv = 2.0 * av * d + lv;   // db_q / dz_v
      if (WJ) a.jv[a.jbase[q] + (t - t0)] = dv;
      if (WJV) jvv = jvv + dv * a.vn[col];
      if (WJTV) a.ojtv[col] = a.ojtv[col] + wq * dv;
      if (av != 0.0) {  // the squared term's diagonal, in node 0's or node N's X block
        const double h2 = 2.0 * av * yq;
        if (WH) {
          const int64_t slot = (fin ? a.N * a.hx : 0) + a.hdiag[k];
          a.hv[slot] = a.hv[slot] + h2;
        }
        if (WHV) a.ohv[col] = a.ohv[col] + h2 * a.vn[col];
      }
    }
    if (WC) a.c[row] = cv - br[q];
    if (WJV) a.ojv[row] = jvv;
  }
}

static ocp_status bin_fill(const ocp* h, BinArgs& a) {
  const Pattern& P = h->pat;
  memset(&a, 0, sizeof(a));
  if (P.nx > 256) return OCP_EDIM;
  a.boff = h->d_boff; a.bv = h->d_bv; a.bcoef = h->d_bcoef; a.jbase = h->d_bbase;
  a.N = h->N;
  a.brow0 = P.nb + (int64_t)h->nx * h->N + (int64_t)P.npath * P.nun;
  a.xN = (int64_t)h->nx * h->N;
  a.nx = h->nx; a.nbin = P.nbin; a.hx = P.hx;
  for (int q = 0; q < P.nbin; ++q) a.nterms += (int)P.bsupp[q].size();
  for (int k = 0; k < P.nx; ++k) a.hdiag[k] = (int16_t)P.hdiag[k];
  return OCP_OK;
}

template <bool WC, bool WJ, bool WH, bool WJV, bool WJTV, bool WHV>
static cudaError_t bin_go(const BinArgs& a, cudaStream_t s) {
  k_bin<WC, WJ, WH, WJV, WJTV, WHV><<<1, 32, 0, s>>>(a);
  return cudaGetLastError();
}

ocp_status bin_eval(ocp* h, unsigned out, const EvalCall& c, cudaStream_t s) {
  (void)out;
  if (h->pat.nbin == 0) return OCP_OK;
  if (c.range) return set_err(h, OCP_EMODEL, "node ranges are not provided with boundary inequalities");
  BinArgs a;
  if (bin_fill(h, a) != OCP_OK) return set_err(h, OCP_EDIM, "too many states for boundary inequalities");
  a.x = c.x; a.y = c.y; a.vn = c.vn; a.vm = c.vm;
  a.c = c.c; a.jv = c.jv; a.hv = c.hv; a.ojv = c.ojv; a.ojtv = c.ojtv; a.ohv = c.ohv;
  const bool C = c.c, J = c.jv, H = c.hv, JV = c.ojv, JT = c.ojtv, HV = c.ohv;
  cudaError_t e = cudaSuccess;
  if (JV || JT || HV) {  // the fused step: every output
    e = bin_go<true, true, true, true, true, true>(a, s);
  } else {
    if (C && e == cudaSuccess) e = bin_go<true, false, false, false, false, false>(a, s);
    if (J && e == cudaSuccess) e = bin_go<false, true, false, false, false, false>(a, s);
    if (H && e == cudaSuccess) e = bin_go<false, false, true, false, false, false>(a, s);
  }
  return cuda_err(h, e, "boundary inequality launch");
}

ocp_status bin_prod(ocp* h, const ProdCall& c, cudaStream_t s) {
  if (h->pat.nbin == 0) return OCP_OK;
  BinArgs a;
  if (bin_fill(h, a) != OCP_OK) return set_err(h, OCP_EDIM, "too many states for boundary inequalities");
  a.x = c.x; a.y = c.y;
  cudaError_t e;
  if (c.kind == P_JPROD) { a.vn = c.v; a.ojv = c.out; e = bin_go<false, false, false, true, false, false>(a, s); }
  else if (c.kind == P_JTPROD) { a.vm = c.v; a.ojtv = c.out; e = bin_go<false, false, false, false, true, false>(a, s); }
  else { a.vn = c.v; a.ohv = c.out; e = bin_go<false, false, false, false, false, true>(a, s); }
  return cuda_err(h, e, "boundary inequality launch");
}

// Device tables of the boundary inequalities (terms, coefficients, slot bases); called after
// every pattern rebuild.
ocp_status bin_upload(ocp* h) {
  cudaFree(h->d_boff); cudaFree(h->d_bv); cudaFree(h->d_bcoef); cudaFree(h->d_bbase);
  h->d_boff = nullptr; h->d_bv = nullptr; h->d_bcoef = nullptr; h->d_bbase = nullptr;
  const Pattern& P = h->pat;
  const int bz = 2 * P.nx;
  std::vector<int32_t> boff(1, 0), bv;
  std::vector<double> coef;
  for (int q = 0; q < P.nbin; ++q) {
    for (int v : P.bsupp[q]) {
      bv.push_back(v);
      coef.push_back(h->bin_a[q * bz + v]);
      coef.push_back(h->bin_b[q * bz + v]);
      coef.push_back(h->bin_l[q * bz + v]);
    }
    boff.push_back((int32_t)bv.size());
  }
  for (int q = 0; q < P.nbin; ++q) coef.push_back(h->bin_r[q]);
  std::vector<int64_t> base(P.jbbase);
  base.insert(base.end(), P.kbbase.begin(), P.kbbase.end());
  if (bv.empty()) bv.push_back(0);
  if (coef.empty()) coef.push_back(0.0);
  cudaError_t e;
  if ((e = ocpg::dev_malloc(&h->d_boff, boff.size() * 4)) != cudaSuccess ||
      (e = ocpg::dev_malloc(&h->d_bv, bv.size() * 4)) != cudaSuccess ||
      (e = ocpg::dev_malloc(&h->d_bcoef, coef.size() * 8)) != cudaSuccess ||
      (e = ocpg::dev_malloc(&h->d_bbase, base.size() * 8)) != cudaSuccess)
    return cuda_err(h, e, "cudaMalloc(boundary inequality tables)");
  if ((e = ocpg::dev_upload(h->d_boff, boff.data(), boff.size() * 4)) != cudaSuccess ||
      (e = ocpg::dev_upload(h->d_bv, bv.data(), bv.size() * 4)) != cudaSuccess ||
      (e = ocpg::dev_upload(h->d_bcoef, coef.data(), coef.size() * 8)) != cudaSuccess ||
      (e = ocpg::dev_upload(h->d_bbase, base.data(), base.size() * 8)) != cudaSuccess)
    return cuda_err(h, e, "cudaMemcpy(boundary inequality tables)");
  return OCP_OK;
}

// ======================================================================================
// Boundary cost (paper Sec. 3, the Bolza term g(X_0, X_N)) added to the objective:
//     g(z) = sum_v [ a_v (z_v - b_v)^2 + l_v z_v ],   z = (X_0, X_N),
// dg/dz_v = 2 a_v (z_v - b_v) + l_v,  d2g/dz_v^2 = 2 a_v (sigma times that in H).  One thread,
// after the model's kernel and the constraint rows' kernels on the same stream: it adds g to
// f, its gradient to g, sigma 2 a_v to the Hessian diagonals of nodes 0 and N and
// sigma 2 a_v v_z to H v, in term order.
// ======================================================================================
struct BolArgs {
  const double* __restrict__ x;
  const double* __restrict__ vn;
  double *f, *g, *hv, *ohv;
  double sigma;
  int64_t N, xN;
  int nx, nt, hx;
  int16_t v[256];         // terms: local index of z (v < nx: X_0, else X_N)
  int16_t hd[256];        // position of (k, k) in the node's X block
  double a[256], b[256], l[256];
};

template <bool WF, bool WG, bool WH, bool WHV>
__global__ void __launch_bounds__(32) k_bol(const __grid_constant__ BolArgs a) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double gs = 0.0;
  for (int t = 0; t < a.nt; ++t) {
    const int v = a.v[t];
    const bool fin = v >= a.nx;
    const int k = fin ? v - a.nx : v;
    const int64_t col = fin ? a.xN + k : (int64_t)k;
    const double z = a.x[col];
    const double d = z - a.b[t];
    if (WF) gs = gs + (a.a[t] * d * d + a.l[t] * z);
    if (WG) a.g[col] = a.g[col] + (2.0 * a.a[t] * d + a.l[t]);
    if (a.a[t] != 0.0) {
      const double h2 = a.sigma * (2.0 * a.a[t]);
      if (WH) {
        const int64_t slot = (fin ? a.N * a.hx : 0) + a.hd[k];
        a.hv[slot] = a.hv[slot] + h2;
      }
      if (WHV) a.ohv[col] = a.ohv[col] + h2 * a.vn[col];
    }
  }
  if (WF) a.f[0] = a.f[0] + gs;
}

static ocp_status bol_fill(const ocp* h, double sigma, BolArgs& a) {
  const Pattern& P = h->pat;
  memset(&a, 0, sizeof(a));
  if (2 * h->nx > 256) return OCP_EDIM;
  a.sigma = sigma; a.N = h->N; a.xN = (int64_t)h->nx * h->N; a.nx = h->nx; a.hx = P.hx;
  for (int v = 0; v < 2 * h->nx; ++v) {
    if (h->bol_a[v] == 0.0 && h->bol_l[v] == 0.0) continue;
    a.v[a.nt] = (int16_t)v;
    a.a[a.nt] = h->bol_a[v]; a.b[a.nt] = h->bol_b[v]; a.l[a.nt] = h->bol_l[v];
    ++a.nt;
  }
  for (int k = 0; k < h->nx; ++k) a.hd[k] = (int16_t)P.hdiag[k];
  return OCP_OK;
}

ocp_status bol_eval(ocp* h, const EvalCall& c, cudaStream_t s) {
  if (!h->has_bol) return OCP_OK;
  if (c.range) return set_err(h, OCP_EMODEL, "node ranges are not provided with a boundary cost");
  BolArgs a;
  if (bol_fill(h, c.sigma, a) != OCP_OK) return set_err(h, OCP_EDIM, "too many states for the boundary cost");
  a.x = c.x; a.vn = c.vn; a.f = c.f; a.g = c.g; a.hv = c.hv; a.ohv = c.ohv;
  const bool F = c.f, G = c.g, H = c.hv, HV = c.ohv;
  if (F && G && H && HV) k_bol<true, true, true, true><<<1, 32, 0, s>>>(a);
  else {
    if (F) k_bol<true, false, false, false><<<1, 32, 0, s>>>(a);
    if (G) k_bol<false, true, false, false><<<1, 32, 0, s>>>(a);
    if (H) k_bol<false, false, true, false><<<1, 32, 0, s>>>(a);
    if (HV) k_bol<false, false, false, true><<<1, 32, 0, s>>>(a);
  }
  return cuda_err(h, cudaGetLastError(), "boundary cost launch");
}

ocp_status bol_prod(ocp* h, const ProdCall& c, cudaStream_t s) {
  if (!h->has_bol || c.kind != P_HPROD) return OCP_OK;
  BolArgs a;
  if (bol_fill(h, c.sigma, a) != OCP_OK) return set_err(h, OCP_EDIM, "too many states for the boundary cost");
  a.x = c.x; a.vn = c.v; a.ohv = c.out;
  k_bol<false, false, false, true><<<1, 32, 0, s>>>(a);
  return cuda_err(h, cudaGetLastError(), "boundary cost launch");
}

}  // namespace ocpg
