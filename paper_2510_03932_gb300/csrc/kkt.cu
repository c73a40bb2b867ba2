// KKT assembly for the interior-point step (paper Sec. 6: the solver assembles the KKT system
// in device buffers from the derivative values of every iteration):
//
//     K = [ H + diag(sigma_x + delta_w)                ]     (lower triangle, COO sorted by
//         [ J                          -delta_c I      ]      (row, col), 0-based)
//
// from the COO values of hess_coo_values and jac_coo_values.  The layout is fixed by the
// pattern compiler: the rows of the (1,1) block node by node (X rows, then U rows, then the
// free final time), then the constraint rows; every row ends with its diagonal, which is
// added where H has none.  One thread per KKT slot decodes its source from the templates, so
// consecutive threads read and write consecutive addresses (a gather with no index array).
#include <algorithm>
#include <cstring>

#include "ocp_internal.h"

namespace ocpg {

constexpr int KKT_TMAX = 256;   // entries of a node's X or U row template (with added diagonals)

struct KktArgs {
  const double* __restrict__ hv;
  const double* __restrict__ jv;
  const double* __restrict__ sx;   // sigma_x (length n) or null
  double* out;
  int32_t* rows;
  int32_t* cols;
  const int64_t* kcbase;   // KKT slots of the defect rows of each component (nx + 1)
  const int64_t* jbase;    // COO slots of the defect rows of each component (nx + 1)
  const int32_t* tmpl;     // Jacobian row templates (RT_STRIDE ints per component)
  const int32_t* fin;      // components of the final rows
  const int32_t* tcol;     // tf-row columns
  int64_t N, n, m, nb, uoff, hbase_u, hbase_t, kb_u, kb_t, kb_c, nnzk;
  double dw, dc;
  int nx, nu, hx, hu, tx, tu, kx, ku, free_tf;
  int16_t ksrc[2 * KKT_TMAX];  // X template then U template: source position or -1
  int16_t ka[2 * KKT_TMAX], kb[2 * KKT_TMAX];
};

__device__ __forceinline__ int64_t kkt_col(const KktArgs& a, int64_t j, int v) {
  return v < a.nx ? (int64_t)a.nx * j + v : a.uoff + (int64_t)a.nu * j + (v - a.nx);
}

// last component k with kcbase[k] <= s
__device__ __forceinline__ int kkt_comp(const KktArgs& a, int64_t s) {
  int lo = 0, hi = a.nx - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.kcbase[mid] <= s) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <bool VALUES>
__global__ void k_kkt(const __grid_constant__ KktArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < a.nnzk; s += stride) {
    double v = 0.0;
    int64_t row = 0, col = 0;
    bool diag = false;          // (1,1)-block diagonal: add sigma_x + delta_w
    if (s < a.kb_t) {           // node rows of the (1,1) block
      const bool xs = s < a.kb_u;
      const int kt = xs ? a.kx : a.ku;
      const int64_t rel = xs ? s : s - a.kb_u;
      const int64_t j = rel / kt;
      const int p = (int)(rel - j * kt) + (xs ? 0 : KKT_TMAX);
      const int src = a.ksrc[p];
      row = kkt_col(a, j, a.ka[p]);
      col = kkt_col(a, j, a.kb[p]);
      diag = a.ka[p] == a.kb[p];
      if (VALUES && src >= 0) v = __ldg(a.hv + (xs ? (int64_t)a.hx * j : a.hbase_u + (int64_t)a.hu * j) + src);
    } else if (s < a.kb_c) {    // the free final time's row: H's tf row, then its diagonal
      const int64_t r = s - a.kb_t, tlen = (int64_t)(a.tx + a.tu) * (a.N + 1);
      row = a.n - 1;
      if (r < tlen) {
        if (VALUES) v = __ldg(a.hv + a.hbase_t + r);
        if (!VALUES) {
          const int64_t xpart = (a.N + 1) * a.tx;
          int64_t j;
          int e;
          if (r < xpart) { j = r / a.tx; e = (int)(r - j * a.tx); }
          else { j = (r - xpart) / a.tu; e = a.tx + (int)(r - xpart - j * a.tu); }
          col = kkt_col(a, j, a.tcol[e]);
        }
      } else {
        col = a.n - 1;
        diag = true;
      }
    } else if (s < a.kcbase[0]) {  // boundary rows: the unit entry, then -delta_c
      const int64_t r = (s - a.kb_c) >> 1;
      row = a.n + r;
      if ((s - a.kb_c) & 1) {
        col = row;
        v = -a.dc;
      } else {
        col = (r < a.nx) ? r : (int64_t)a.nx * a.N + a.fin[r - a.nx];
        if (VALUES) v = __ldg(a.jv + r);
      }
    } else {                       // defect rows: the Jacobian row, then -delta_c
      const int k = kkt_comp(a, s);
      const int32_t* t = a.tmpl + RT_STRIDE * k;
      const int rx = t[0], ru = t[1];
      const int cnt = 2 * (rx + ru) + a.free_tf;
      const int64_t rel = s - a.kcbase[k];
      const int64_t j = rel / (cnt + 1);
      const int e = (int)(rel - j * (cnt + 1));
      row = a.n + a.nb + (int64_t)k * a.N + j;
      if (e == cnt) {
        col = row;
        v = -a.dc;
      } else {
        if (VALUES) v = __ldg(a.jv + a.jbase[k] + j * cnt + e);
        if (!VALUES) {
          if (e == 2 * (rx + ru)) col = a.n - 1;
          else if (e < rx) col = (int64_t)a.nx * j + t[2 + e];
          else if (e < 2 * rx) col = (int64_t)a.nx * (j + 1) + t[2 + (e - rx)];
          else if (e < 2 * rx + ru) col = a.uoff + (int64_t)a.nu * j + t[2 + RT_XV + (e - 2 * rx)];
          else col = a.uoff + (int64_t)a.nu * (j + 1) + t[2 + RT_XV + (e - 2 * rx - ru)];
        }
      }
    }
    if (VALUES) {
      if (diag) v = v + ((a.sx ? __ldg(a.sx + row) : 0.0) + a.dw);
      a.out[s] = v;
    } else {
      a.rows[s] = (int32_t)row;
      a.cols[s] = (int32_t)col;
    }
  }
}

static ocp_status kkt_fill(const ocp* h, KktArgs& a) {
  const Pattern& P = h->pat;
  if (P.nnzk < 0) return OCP_EDIM;
  if ((int)P.kxt.size() > KKT_TMAX || (int)P.kut.size() > KKT_TMAX) return OCP_EDIM;
  memset(&a, 0, sizeof(a));
  a.kcbase = h->d_kcbase; a.jbase = h->d_jbase; a.tmpl = h->d_rowtmpl; a.fin = h->d_fin; a.tcol = h->d_tcol;
  a.N = h->N; a.n = P.n; a.m = P.m; a.nb = P.nb; a.uoff = (int64_t)h->nx * (h->N + 1);
  a.hbase_u = P.hbase_u; a.hbase_t = P.hbase_t;
  a.kb_u = P.kb_u; a.kb_t = P.kb_t; a.kb_c = P.kb_c; a.nnzk = P.nnzk;
  a.nx = h->nx; a.nu = h->nu; a.hx = P.hx; a.hu = P.hu; a.tx = P.tx; a.tu = P.tu;
  a.kx = (int)P.kxt.size(); a.ku = (int)P.kut.size(); a.free_tf = P.free_tf;
  for (int i = 0; i < a.kx; ++i) { a.ksrc[i] = (int16_t)P.kxt[i].src; a.ka[i] = (int16_t)P.kxt[i].a; a.kb[i] = (int16_t)P.kxt[i].b; }
  for (int i = 0; i < a.ku; ++i) {
    a.ksrc[KKT_TMAX + i] = (int16_t)P.kut[i].src;
    a.ka[KKT_TMAX + i] = (int16_t)P.kut[i].a;
    a.kb[KKT_TMAX + i] = (int16_t)P.kut[i].b;
  }
  return OCP_OK;
}

static int kkt_grid(const ocp* h, int64_t nnz) {
  const int64_t blocks = std::min<int64_t>((nnz + 255) / 256, (int64_t)h->num_sms * 16);
  return (int)std::max<int64_t>(blocks, 1);
}

}  // namespace ocpg

using namespace ocpg;

extern "C" {

ocp_status ocp_kkt_dims(const ocp_t* h, int64_t* nnzk) {
  if (!h || !nnzk) return OCP_EINVAL;
  if (h->pat.nnzk < 0) return OCP_EDIM;
  *nnzk = h->pat.nnzk;
  return OCP_OK;
}

ocp_status ocp_kkt_structure(ocp_t* h, int32_t* rows, int32_t* cols, void* stream) {
  if (!h) return OCP_EINVAL;
  if (!rows || !cols) return set_err(h, OCP_EINVAL, "rows and cols are required");
  KktArgs a;
  if (kkt_fill(h, a) != OCP_OK) return set_err(h, OCP_EDIM, "KKT matrix too large for the int32 interface");
  a.rows = rows; a.cols = cols;
  k_kkt<false><<<kkt_grid(h, a.nnzk), 256, 0, (cudaStream_t)stream>>>(a);
  return cuda_err(h, cudaGetLastError(), "KKT structure launch");
}

ocp_status ocp_kkt_values(ocp_t* h, const double* hvals, const double* jvals, const double* sigma_x,
                          double delta_w, double delta_c, double* kvals, void* stream) {
  if (!h) return OCP_EINVAL;
  if (!hvals || !jvals || !kvals) return set_err(h, OCP_EINVAL, "hvals, jvals and kvals are required");
  if (((uintptr_t)hvals | (uintptr_t)jvals | (uintptr_t)kvals | (uintptr_t)sigma_x) & 7u)
    return set_err(h, OCP_EINVAL, "arrays must be 8-byte aligned");
  KktArgs a;
  if (kkt_fill(h, a) != OCP_OK) return set_err(h, OCP_EDIM, "KKT matrix too large for the int32 interface");
  a.hv = hvals; a.jv = jvals; a.sx = sigma_x; a.out = kvals; a.dw = delta_w; a.dc = delta_c;
  k_kkt<true><<<kkt_grid(h, a.nnzk), 256, 0, (cudaStream_t)stream>>>(a);
  return cuda_err(h, cudaGetLastError(), "KKT values launch");
}

}  // extern "C"
