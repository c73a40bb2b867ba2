// Host pattern compiler and the COO structure kernels.
//
// The transcription (paper Sec. 5) makes, for every state component k, one defect row per
// interval j; row (k, j) touches only z_j and z_{j+1}.  The pattern compiler turns the
// model's per-node templates into the slot layout of the COO arrays:
//   Jacobian:  [nb boundary rows, 1 entry each] then, component by component, N rows of
//              count_k entries; row (k, j) starts at jbase[k] + j*count_k and lists, by
//              increasing column, its entries on X_j, X_{j+1}, U_j, U_{j+1}.
//   Hessian:   block-diagonal by node (the defects are sums of one-node terms and the cost is
//              a sum over nodes): the hx X-row entries of every node in node order, then the
//              hu U-row entries of every node; within a node, by (row, col).
//   Free final time tf (the last unknown): every defect row ends with its tf entry, and the
//              Hessian ends with the tf row (tf against the state columns of every node, then
//              the control columns; no (tf, tf) entry: c and F are linear in tf).
//   Final rows may cover a subset of the components (nb = nx + their count).
// Sorting by (row, col) globally gives exactly this order because X columns precede U columns.
#include <algorithm>
#include <cstring>

#include "models.cuh"
#include "node_kernels.cuh"
#include "ocp_internal.h"

namespace ocpg {

template <class M>
static void rows_from(std::vector<RowTemplate>& rows) {
  static_assert(M::MAXRX <= RT_XV && M::MAXRU <= RT_UV, "row template wider than the device table");
  rows.assign(M::NX, RowTemplate());
  for (int k = 0; k < M::NX; ++k) {
    rows[k].rx = M::RX(k);
    rows[k].ru = M::RU(k);
    for (int e = 0; e < M::RX(k); ++e) { rows[k].xv[e] = M::XV(k, e); rows[k].jz[e] = M::JZ(k, e); }
    for (int e = 0; e < M::RU(k); ++e) rows[k].uv[e] = M::UV(k, e);
  }
}

void model_row_templates(int model, int nx, std::vector<RowTemplate>& rows) {
  switch (model) {
    case OCP_MODEL_VDP: rows_from<VdP>(rows); break;
    case OCP_MODEL_CARTPOLE: rows_from<CartPole>(rows); break;
    case OCP_MODEL_DINT: rows_from<Dint>(rows); break;
    case OCP_MODEL_QUADROTOR: rows_from<Quadrotor>(rows); break;
    case OCP_MODEL_GODDARD: rows_from<Goddard>(rows); break;
    case OCP_MODEL_HEAT1D:
      rows.assign(nx, RowTemplate());
      for (int k = 0; k < nx; ++k) {
        RowTemplate& r = rows[k];
        r.rx = 0;
        if (k > 0) r.xv[r.rx++] = k - 1;
        r.xv[r.rx++] = k;
        if (k < nx - 1) r.xv[r.rx++] = k + 1;
        r.ru = (k == 0) ? 1 : 0;
        r.uv[0] = (k == 0) ? 0 : -1;
      }
      break;
    default: rows.clear();
  }
}

template <class M>
static void hmax_from(std::vector<std::pair<int, int>>& ent, std::vector<int>& is_dyn) {
  constexpr HTmpl<M> HT{};
  ent.clear();
  is_dyn.clear();
  for (int e = 0; e < HT.n; ++e) {
    ent.push_back({HT.a[e], HT.b[e]});
    is_dyn.push_back(HT.dyn[e] >= 0 ? 1 : 0);
  }
}

void model_hess_max_template(int model, int nx, std::vector<std::pair<int, int>>& ent, std::vector<int>& is_dyn) {
  switch (model) {
    case OCP_MODEL_VDP: hmax_from<VdP>(ent, is_dyn); break;
    case OCP_MODEL_CARTPOLE: hmax_from<CartPole>(ent, is_dyn); break;
    case OCP_MODEL_DINT: hmax_from<Dint>(ent, is_dyn); break;
    case OCP_MODEL_QUADROTOR: hmax_from<Quadrotor>(ent, is_dyn); break;
    case OCP_MODEL_GODDARD: hmax_from<Goddard>(ent, is_dyn); break;
    case OCP_MODEL_HEAT1D:
      ent.clear();
      is_dyn.clear();
      for (int k = 0; k < nx; ++k) { ent.push_back({k, k}); is_dyn.push_back(1); }
      ent.push_back({nx, nx});
      is_dyn.push_back(0);
      break;
    default: ent.clear(); is_dyn.clear();
  }
}

bool build_pattern(ocp* h, std::string& why) {
  Pattern& P = h->pat;
  P = Pattern();
  P.nx = h->nx; P.nu = h->nu; P.nz = h->nx + h->nu; P.N = h->N;
  P.free_tf = h->free_tf ? 1 : 0;
  P.scheme = h->scheme;
  P.nun = (P.scheme == OCP_SCHEME_EULER) ? P.N : P.N + 1;
  P.n = (int64_t)P.nx * (P.N + 1) + (int64_t)P.nu * P.nun + P.free_tf;
  P.npath = h->npath;
  P.nbin = h->nbin;
  if (h->has_final) {
    if (h->fin_comp.empty()) for (int k = 0; k < P.nx; ++k) P.fin.push_back(k);
    else P.fin = h->fin_comp;
  }
  P.nb = (int64_t)P.nx + (int64_t)P.fin.size();
  P.m = P.nb + (int64_t)P.nx * P.N + (int64_t)P.npath * P.nun + P.nbin;
  model_row_templates(h->model, h->nx, P.rows);
  if ((int)P.rows.size() != P.nx) { why = "no row template for this model"; return false; }
  P.jbase.assign(P.nx + 1, 0);
  P.jbase[0] = P.nb;
  for (int k = 0; k < P.nx; ++k) P.jbase[k + 1] = P.jbase[k] + (int64_t)P.row_count(k) * P.N;
  P.nnzj = P.jbase[P.nx];
  // path rows after the defect rows: one entry per variable of the row's support
  P.psupp.assign(P.npath, std::vector<int>());
  P.jpbase.assign(P.npath + 1, P.nnzj);
  for (int p = 0; p < P.npath; ++p) {
    for (int v = 0; v < P.nz; ++v)
      if (h->path_a[p * P.nz + v] != 0.0 || h->path_l[p * P.nz + v] != 0.0) P.psupp[p].push_back(v);
    P.jpbase[p + 1] = P.jpbase[p] + (int64_t)P.psupp[p].size() * P.nun;
  }
  P.nnzj = P.jpbase[P.npath];
  // boundary-inequality rows after the path rows: one entry per variable of (X_0, X_N) in the
  // row's support, X_0 columns before X_N columns
  const int bz = 2 * P.nx;
  P.bsupp.assign(P.nbin, std::vector<int>());
  P.jbbase.assign(P.nbin + 1, P.nnzj);
  for (int q = 0; q < P.nbin; ++q) {
    for (int v = 0; v < bz; ++v)
      if (h->bin_a[q * bz + v] != 0.0 || h->bin_l[q * bz + v] != 0.0) P.bsupp[q].push_back(v);
    P.jbbase[q + 1] = P.jbbase[q] + (int64_t)P.bsupp[q].size();
  }
  P.nnzj = P.jbbase[P.nbin];
  std::vector<std::pair<int, int>> ent;
  std::vector<int> dyn;
  model_hess_max_template(h->model, h->nx, ent, dyn);
  P.hpos.assign(ent.size(), (int8_t)-1);
  int px = 0, pu = 0;
  std::vector<std::pair<int, int>> ex, eu;
  for (size_t e = 0; e < ent.size(); ++e) {
    const int a = ent[e].first, b = ent[e].second;
    const double coef = a < P.nx ? h->q[a] : h->r[a - P.nx];
    bool path_sq = false;  // a squared path or boundary term needs the diagonal
    for (int p = 0; p < P.npath && a == b; ++p) path_sq = path_sq || h->path_a[p * P.nz + a] != 0.0;
    // (one template for every node: a boundary term's diagonal is present at every node)
    for (int q = 0; q < P.nbin && a == b && a < P.nx; ++q)
      path_sq = path_sq || h->bin_a[q * bz + a] != 0.0 || h->bin_a[q * bz + P.nx + a] != 0.0;
    if (h->has_bol && a == b && a < P.nx)  // the boundary cost's squared terms likewise
      path_sq = path_sq || h->bol_a[a] != 0.0 || h->bol_a[P.nx + a] != 0.0;
    const bool present = dyn[e] || (a == b && (coef != 0.0 || path_sq));
    if (!present) continue;
    if (a < P.nx) { P.hpos[e] = (int8_t)(px < 127 ? px : 127); ++px; ex.push_back(ent[e]); }
    else { P.hpos[e] = (int8_t)pu; ++pu; eu.push_back(ent[e]); }
  }
  P.hx = px;
  P.hu = pu;
  P.hent = ex;
  P.hent.insert(P.hent.end(), eu.begin(), eu.end());
  P.hdiag.assign(P.nz, -1);
  for (int e = 0; e < P.hx; ++e)
    if (P.hent[e].first == P.hent[e].second) P.hdiag[P.hent[e].first] = e;
  for (int e = 0; e < P.hu; ++e)
    if (P.hent[P.hx + e].first == P.hent[P.hx + e].second) P.hdiag[P.hent[P.hx + e].first] = e;
  P.hbase_u = (int64_t)P.hx * P.nun;
  P.nnzh = (int64_t)(P.hx + P.hu) * P.nun;
  if (P.free_tf) {
    // tf row: the columns where some f_k has a derivative, and the cost columns
    std::vector<bool> col(P.nz, false);
    for (int k = 0; k < P.nx; ++k) {
      for (int e = 0; e < P.rows[k].rx; ++e)
        if (!P.rows[k].jz[e]) col[P.rows[k].xv[e]] = true;
      for (int e = 0; e < P.rows[k].ru; ++e) col[P.nx + P.rows[k].uv[e]] = true;
    }
    for (int v = 0; v < P.nz; ++v)
      if ((v < P.nx ? h->q[v] : h->r[v - P.nx]) != 0.0) col[v] = true;
    for (int v = 0; v < P.nz; ++v)
      if (col[v]) { P.tcol.push_back(v); if (v < P.nx) ++P.tx; else ++P.tu; }
    P.hbase_t = P.nnzh;
    P.nnzh += (int64_t)(P.tx + P.tu) * P.nun;
  }
  // KKT layout: rows of the (1,1) block node by node (X rows, then U rows), the tf row, then
  // the constraint rows, each with its diagonal last (the largest column of a lower row)
  for (int a = 0; a < P.nz; ++a) {
    std::vector<Pattern::KEnt>& t = (a < P.nx) ? P.kxt : P.kut;
    const int base = (a < P.nx) ? 0 : P.hx;
    bool diag = false;
    for (int e = (a < P.nx ? 0 : P.hx); e < (a < P.nx ? P.hx : P.hx + P.hu); ++e)
      if (P.hent[e].first == a) {
        t.push_back({e - base, a, P.hent[e].second});
        diag = diag || (P.hent[e].second == a);
      }
    if (!diag) t.push_back({-1, a, a});
  }
  // (Euler: the X rows of node N carry only their diagonal)
  P.kb_u = (int64_t)P.kxt.size() * P.nun + (P.scheme == OCP_SCHEME_EULER ? P.nx : 0);
  P.kb_t = P.kb_u + (int64_t)P.kut.size() * P.nun;
  P.kb_c = P.kb_t + (P.free_tf ? (int64_t)(P.tx + P.tu) * P.nun + 1 : 0);
  P.kcbase.assign(P.nx + 1, 0);
  P.kcbase[0] = P.kb_c + 2 * P.nb;
  for (int k = 0; k < P.nx; ++k) P.kcbase[k + 1] = P.kcbase[k] + (int64_t)(P.row_count(k) + 1) * P.N;
  P.kpbase.assign(P.npath + 1, P.kcbase[P.nx]);
  for (int p = 0; p < P.npath; ++p) P.kpbase[p + 1] = P.kpbase[p] + (int64_t)(P.psupp[p].size() + 1) * P.nun;
  P.kbbase.assign(P.nbin + 1, P.kpbase[P.npath]);
  for (int q = 0; q < P.nbin; ++q) P.kbbase[q + 1] = P.kbbase[q] + (int64_t)P.bsupp[q].size() + 1;
  P.nnzk = P.kbbase[P.nbin];
  const int64_t lim = (int64_t)1 << 31;
  if (P.nnzk >= lim || P.n + P.m >= lim) P.nnzk = -1;
  if (P.n >= lim || P.m >= lim || P.nnzj >= lim || P.nnzh >= lim || fault_dims()) {
    why = "problem too large for the int32 COO interface (n, m or nnz >= 2^31)";
    return false;
  }
  return true;
}

// ---------------------------------------------------------------------------------------
// Structure kernels: one thread per slot, decoding (row, col) from the templates.
// ---------------------------------------------------------------------------------------
struct JacStructArgs {
  int32_t* rows;
  int32_t* cols;
  const int32_t* tmpl;   // per component (RT_STRIDE ints): rx, ru, xv[RT_XV], uv[RT_UV]
  const int64_t* jbase;  // nx + 1
  const int32_t* fin;    // components of the final rows
  const int64_t* pbase;  // path rows: first slot of row p (npath + 1)
  const int32_t* poff;   // path rows: support of row p = pv[poff[p] .. poff[p+1])
  const int32_t* pv;
  const int64_t* bbase;  // boundary-inequality rows: first slot of row q (nbin + 1)
  const int32_t* boff;   // their supports: bv[boff[q] .. boff[q+1]) (local indices of (X_0, X_N))
  const int32_t* bv;
  int64_t N, nb, nnzj, uoff, n, nun, prow0;   // prow0: first path row
  int nx, nu, free_tf, euler, npath, nbin;
};

__global__ void k_jac_structure(const __grid_constant__ JacStructArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < a.nnzj; s += stride) {
    int64_t row, col;
    if (s < a.nb) {
      row = s;
      col = (s < a.nx) ? s : (int64_t)a.nx * a.N + a.fin[s - a.nx];
    } else if (a.nbin > 0 && s >= a.bbase[0]) {  // boundary-inequality rows
      int q = 0;
      while (q + 1 < a.nbin && a.bbase[q + 1] <= s) ++q;
      const int v = a.bv[a.boff[q] + (int)(s - a.bbase[q])];
      row = a.prow0 + (int64_t)a.npath * a.nun + q;
      col = v < a.nx ? v : (int64_t)a.nx * a.N + (v - a.nx);
    } else if (a.npath > 0 && s >= a.pbase[0]) {  // path rows
      int p = 0;
      while (p + 1 < a.npath && a.pbase[p + 1] <= s) ++p;
      const int cnt = a.poff[p + 1] - a.poff[p];
      const int64_t rel = s - a.pbase[p];
      const int64_t i = rel / cnt;
      const int v = a.pv[a.poff[p] + (int)(rel - i * cnt)];
      row = a.prow0 + (int64_t)p * a.nun + i;
      col = v < a.nx ? (int64_t)a.nx * i + v : a.uoff + (int64_t)a.nu * i + (v - a.nx);
    } else {
      int lo = 0, hi = a.nx - 1;  // last component with jbase <= s
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.jbase[mid] <= s) lo = mid; else hi = mid - 1;
      }
      const int k = lo;
      const int32_t* t = a.tmpl + RT_STRIDE * k;
      const int rx = t[0], ru = t[1];
      const int cnt = a.euler ? rx + 1 + ru : 2 * (rx + ru) + a.free_tf;
      const int64_t rel = s - a.jbase[k];
      const int64_t j = rel / cnt;
      const int e = (int)(rel - j * cnt);
      row = a.nb + (int64_t)k * a.N + j;
      if (a.euler) {  // X_j template, X_{j+1,k}, U_j template
        if (e < rx) col = (int64_t)a.nx * j + t[2 + e];
        else if (e == rx) col = (int64_t)a.nx * (j + 1) + k;
        else col = a.uoff + (int64_t)a.nu * j + t[2 + RT_XV + (e - rx - 1)];
      } else if (e == 2 * (rx + ru)) col = a.n - 1;  // the free final time closes the row
      else if (e < rx) col = (int64_t)a.nx * j + t[2 + e];
      else if (e < 2 * rx) col = (int64_t)a.nx * (j + 1) + t[2 + (e - rx)];
      else if (e < 2 * rx + ru) col = a.uoff + (int64_t)a.nu * j + t[2 + RT_XV + (e - 2 * rx)];
      else col = a.uoff + (int64_t)a.nu * (j + 1) + t[2 + RT_XV + (e - 2 * rx - ru)];
    }
    a.rows[s] = (int32_t)row;
    a.cols[s] = (int32_t)col;
  }
}

struct HessStructArgs {
  int32_t* rows;
  int32_t* cols;
  const int32_t* hent;  // (a, b) pairs: hx X-block entries then hu U-block entries
  const int32_t* tcol;  // tf-row columns: tx state then tu control local indices
  int64_t N, hbase_u, hbase_t, nnzh, uoff, n;
  int nx, nu, hx, hu, tx, tu;
};

__device__ __forceinline__ int64_t local_col(int64_t j, int v, int nx, int nu, int64_t uoff) {
  return v < nx ? (int64_t)nx * j + v : uoff + (int64_t)nu * j + (v - nx);
}

__global__ void k_hess_structure(const __grid_constant__ HessStructArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < a.nnzh; s += stride) {
    int64_t j;
    int e;
    if (s >= a.hbase_t) {  // the tf row: state columns of every node, then control columns
      const int64_t r = s - a.hbase_t, xpart = (a.N + 1) * a.tx;
      if (r < xpart) { j = r / a.tx; e = (int)(r - j * a.tx); }
      else { j = (r - xpart) / a.tu; e = a.tx + (int)(r - xpart - j * a.tu); }
      a.rows[s] = (int32_t)(a.n - 1);
      a.cols[s] = (int32_t)local_col(j, a.tcol[e], a.nx, a.nu, a.uoff);
      continue;
    }
    if (s < a.hbase_u) { j = s / a.hx; e = (int)(s - j * a.hx); }
    else { const int64_t r = s - a.hbase_u; j = r / a.hu; e = a.hx + (int)(r - j * a.hu); }
    const int va = a.hent[2 * e], vb = a.hent[2 * e + 1];
    a.rows[s] = (int32_t)local_col(j, va, a.nx, a.nu, a.uoff);
    a.cols[s] = (int32_t)local_col(j, vb, a.nx, a.nu, a.uoff);
  }
}

ocp_status launch_jac_structure(const ocp* h, int32_t* rows, int32_t* cols, cudaStream_t s) {
  JacStructArgs a;
  a.rows = rows; a.cols = cols; a.tmpl = h->d_rowtmpl; a.jbase = h->d_jbase; a.fin = h->d_fin;
  a.N = h->N; a.nb = h->pat.nb; a.nnzj = h->pat.nnzj; a.uoff = (int64_t)h->nx * (h->N + 1); a.n = h->pat.n;
  a.nx = h->nx; a.nu = h->nu; a.free_tf = h->pat.free_tf; a.euler = h->pat.scheme == OCP_SCHEME_EULER;
  a.pbase = h->d_pbase; a.poff = h->d_poff; a.pv = h->d_pv; a.npath = h->pat.npath;
  a.nun = h->pat.nun; a.prow0 = h->pat.nb + (int64_t)h->nx * h->N;
  a.bbase = h->d_bbase; a.boff = h->d_boff; a.bv = h->d_bv; a.nbin = h->pat.nbin;
  const int64_t blocks = std::min<int64_t>((a.nnzj + 255) / 256, (int64_t)h->num_sms * 16);
  k_jac_structure<<<(int)std::max<int64_t>(blocks, 1), 256, 0, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? OCP_OK : OCP_ECUDA;
}

ocp_status launch_hess_structure(const ocp* h, int32_t* rows, int32_t* cols, cudaStream_t s) {
  HessStructArgs a;
  a.rows = rows; a.cols = cols; a.hent = h->d_hent; a.tcol = h->d_tcol;
  a.N = h->N; a.hbase_u = h->pat.hbase_u; a.nnzh = h->pat.nnzh; a.uoff = (int64_t)h->nx * (h->N + 1);
  a.hbase_t = h->pat.free_tf ? h->pat.hbase_t : h->pat.nnzh;
  a.n = h->pat.n;
  a.nx = h->nx; a.nu = h->nu; a.hx = h->pat.hx; a.hu = h->pat.hu; a.tx = h->pat.tx; a.tu = h->pat.tu;
  const int64_t blocks = std::min<int64_t>((a.nnzh + 255) / 256, (int64_t)h->num_sms * 16);
  k_hess_structure<<<(int)std::max<int64_t>(blocks, 1), 256, 0, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? OCP_OK : OCP_ECUDA;
}

}  // namespace ocpg
