// KKT assembly for the interior-point step (paper Sec. 6: the solver assembles the KKT system
// in device buffers from the derivative values of every iteration):
//
//     K = [ H + diag(sigma_x + delta_w)                ]     (lower triangle, COO sorted by
//         [ J                          -delta_c I      ]      (row, col), 0-based)
//
// from the COO values of hess_coo_values and jac_coo_values.  The layout is fixed by the
// pattern compiler: the rows of the (1,1) block node by node (X rows, then U rows, then the
// free final time), then the constraint rows; every row ends with its diagonal, which is
// added where H has none.  Each KKT slot's source is decoded from the templates (no index
// array is read), so consecutive threads read and write consecutive addresses.
#include <algorithm>
#include <cstring>

#include "ocp_internal.h"

namespace ocpg {

constexpr int KKT_TMAX = 256;   // entries of a node's X or U row template (with added diagonals)
constexpr int KKT_MAXREG = 5 + 128 + 16 + 16;  // X, X_N, U, tf, boundary rows, defect rows per component,
                                                // path rows, boundary-inequality rows

// A run of KKT slots with one layout: slot i of the region is KKT entry out + i; its period is
// the template length (X, U) or the row length plus the diagonal (defects); src / stride give
// the first source value and the source advance per period.
struct KRegion {
  int64_t out, src;
  uint32_t len, period, stride;
  int kind;
  uint32_t block0;   // first block of the values kernel that works on this region
};

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
  const int64_t* kpbase;   // KKT slots of the path rows (npath + 1)
  const int32_t* poff;     // path rows: support of row p = pv[poff[p] .. poff[p+1])
  const int32_t* pv;
  const int64_t* kbbase;   // KKT slots of the boundary-inequality rows (nbin + 1)
  const int32_t* boff;     // their supports: bv[boff[q] .. boff[q+1]) (local indices of (X_0, X_N))
  const int32_t* bv;
  int64_t N, n, m, nb, uoff, hbase_u, hbase_t, kb_xn, kb_u, kb_t, kb_c, nnzk;
  double dw, dc;
  int nx, nu, hx, hu, tx, tu, kx, ku, free_tf, euler, npath, nbin;
  int64_t nun, prow0;
  int16_t ksrc[2 * KKT_TMAX];  // X template then U template: source position or -1
  int16_t ka[2 * KKT_TMAX], kb[2 * KKT_TMAX];
  int nreg;
  uint32_t nblocks;   // blocks of the values kernel
  KRegion reg[KKT_MAXREG];
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

// Values: the KKT is cut into regions of uniform layout (the X rows of the nodes, the U rows,
// the tf row, the boundary rows, the defect rows of each component), each with its own range
// of blocks.  In the row regions a block takes KKT_ROWS consecutive periods (nodes or defect rows)
// and its threads walk the block's output slots in order, so loads and stores are
// coalesced; the period of a slot comes from a single-precision product (exact for the
// block-local indices, see kkt_div) instead of an integer division, and the X / U templates
// sit in shared memory.  Moved values are copied bit for bit; the (1,1) diagonal gets
// sigma_x + delta_w, the constraint diagonal is -delta_c.
constexpr int KKT_ROWS = 1024;
constexpr int KKT_BATCH = 4;
enum { KR_X = 0, KR_U = 1, KR_TF = 2, KR_BND = 3, KR_DEF = 4, KR_XN = 5 };

// floor(i / P) for block-local i < KKT_ROWS * P, P <= 1024: (i + 1/2) / P lies at least 1/(2P) >=
// 2^-11 from an integer; its single-precision value (below KKT_ROWS = 2^10, computed from
// 1/P rounded to nearest and a product rounded toward zero) is off by less than 2^-12.
__device__ __forceinline__ uint32_t kkt_div(uint32_t i, float invP) {
  return (uint32_t)__fmul_rz((float)i + 0.5f, invP);
}

__global__ void __launch_bounds__(256) k_kkt_values(const __grid_constant__ KktArgs a) {
  __shared__ int16_t s_src[KKT_TMAX], s_a[KKT_TMAX];
  __shared__ uint8_t s_diag[KKT_TMAX];
  // the region of this block: the last one whose first block is <= blockIdx.x
  int lo = 0, hi = a.nreg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.reg[mid].block0 <= blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const KRegion R = a.reg[lo];
  const uint32_t chunk = blockIdx.x - R.block0;
  if (R.kind == KR_TF || R.kind == KR_BND || R.kind == KR_XN) {  // short regions: slot by slot
    const uint32_t i1 = min(R.len, (chunk + 1) * 256u * KKT_ROWS);
    for (uint32_t i = chunk * 256u * KKT_ROWS + threadIdx.x; i < i1; i += blockDim.x) {
      double v;
      if (R.kind == KR_TF) {
        if (i + 1 < R.len) v = __ldg(a.hv + R.src + i);
        else v = (a.sx ? __ldg(a.sx + a.n - 1) : 0.0) + a.dw;
      } else if (R.kind == KR_XN) {  // Euler: the X rows of node N hold only their diagonal
        v = (a.sx ? __ldg(a.sx + (int64_t)a.nx * a.N + i) : 0.0) + a.dw;
      } else {
        v = (i & 1) ? -a.dc : __ldg(a.jv + (i >> 1));
      }
      a.out[R.out + i] = v;
    }
    return;
  }
  const uint32_t P = R.period;
  if (R.kind != KR_DEF) {  // the node template of the X or U rows
    const int toff = (R.kind == KR_U) ? KKT_TMAX : 0;
    for (uint32_t p = threadIdx.x; p < P; p += blockDim.x) {
      s_src[p] = a.ksrc[toff + p];
      s_a[p] = a.ka[toff + p];
      s_diag[p] = a.ka[toff + p] == a.kb[toff + p];
    }
    __syncthreads();
  }
  const float invP = 1.0f / (float)P;
  const uint32_t nper = R.len / P;   // nodes or defect rows of the region
  const uint32_t c0 = chunk * KKT_ROWS;
  const uint32_t nloc = min((uint32_t)KKT_ROWS, nper - c0) * P;
  // (the output never aliases the inputs: loads of later slots may be issued before stores)
  const double* __restrict__ src0 = ((R.kind == KR_DEF) ? a.jv : a.hv) + R.src + (int64_t)c0 * R.stride;
  double* __restrict__ out0 = a.out + R.out + (int64_t)c0 * P;
  // KKT_BATCH slots per thread per pass: their loads are issued before any store
  for (uint32_t i0 = threadIdx.x; i0 < nloc; i0 += KKT_BATCH * 256u) {
    double v[KKT_BATCH];
#pragma unroll
    for (int q = 0; q < KKT_BATCH; ++q) {
      const uint32_t i = i0 + q * 256u;
      v[q] = 0.0;
      if (i >= nloc) continue;
      const uint32_t jl = kkt_div(i, invP);
      const uint32_t e = i - jl * P;
      if (R.kind == KR_DEF) {
        v[q] = (e + 1 == P) ? -a.dc : __ldg(src0 + (i - jl));   // i - jl: the diagonals before this slot
      } else {
        const int sp = s_src[e];
        v[q] = (sp >= 0) ? __ldg(src0 + (int64_t)R.stride * jl + sp) : 0.0;
        if (s_diag[e]) {
          const int64_t j = (int64_t)c0 + jl;
          const int64_t row = (R.kind == KR_X) ? (int64_t)a.nx * j + s_a[e] : a.uoff + (int64_t)a.nu * j + (s_a[e] - a.nx);
          v[q] = v[q] + ((a.sx ? __ldg(a.sx + row) : 0.0) + a.dw);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < KKT_BATCH; ++q) {
      const uint32_t i = i0 + q * 256u;
      if (i < nloc) out0[i] = v[q];
    }
  }
}

// Structure: one thread per slot, (row, col) decoded from the same layout.
__global__ void k_kkt_structure(const __grid_constant__ KktArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < a.nnzk; s += stride) {
    int64_t row, col;
    if (s >= a.kb_xn && s < a.kb_u) {  // Euler: diagonal of the X rows of node N
      row = col = (int64_t)a.nx * a.N + (s - a.kb_xn);
    } else if (s < a.kb_t) {    // node rows of the (1,1) block
      const bool xs = s < a.kb_u;
      const int kt = xs ? a.kx : a.ku;
      const int64_t rel = xs ? s : s - a.kb_u;
      const int64_t j = rel / kt;
      const int p = (int)(rel - j * kt) + (xs ? 0 : KKT_TMAX);
      row = kkt_col(a, j, a.ka[p]);
      col = kkt_col(a, j, a.kb[p]);
    } else if (s < a.kb_c) {    // the free final time's row: H's tf row, then its diagonal
      const int64_t r = s - a.kb_t, tlen = (int64_t)(a.tx + a.tu) * (a.N + 1);
      row = a.n - 1;
      if (r < tlen) {
        const int64_t xpart = (a.N + 1) * a.tx;
        int64_t j;
        int e;
        if (r < xpart) { j = r / a.tx; e = (int)(r - j * a.tx); }
        else { j = (r - xpart) / a.tu; e = a.tx + (int)(r - xpart - j * a.tu); }
        col = kkt_col(a, j, a.tcol[e]);
      } else {
        col = a.n - 1;
      }
    } else if (s < a.kcbase[0]) {  // boundary rows: the unit entry, then the diagonal
      const int64_t r = (s - a.kb_c) >> 1;
      row = a.n + r;
      if ((s - a.kb_c) & 1) col = row;
      else col = (r < a.nx) ? r : (int64_t)a.nx * a.N + a.fin[r - a.nx];
    } else if (a.nbin > 0 && s >= a.kbbase[0]) {  // boundary-inequality rows: entries, diagonal
      int q = 0;
      while (q + 1 < a.nbin && a.kbbase[q + 1] <= s) ++q;
      const int cnt = a.boff[q + 1] - a.boff[q];
      const int e = (int)(s - a.kbbase[q]);
      row = a.n + a.prow0 + (int64_t)a.npath * a.nun + q;
      if (e == cnt) col = row;
      else {
        const int v = a.bv[a.boff[q] + e];
        col = v < a.nx ? v : (int64_t)a.nx * a.N + (v - a.nx);
      }
    } else if (a.npath > 0 && s >= a.kpbase[0]) {  // path rows: their entries, then the diagonal
      int p = 0;
      while (p + 1 < a.npath && a.kpbase[p + 1] <= s) ++p;
      const int cnt = a.poff[p + 1] - a.poff[p];
      const int64_t rel = s - a.kpbase[p];
      const int64_t i = rel / (cnt + 1);
      const int e = (int)(rel - i * (cnt + 1));
      row = a.n + a.prow0 + (int64_t)p * a.nun + i;
      col = (e == cnt) ? row : kkt_col(a, i, a.pv[a.poff[p] + e]);
    } else {                       // defect rows: the Jacobian row, then the diagonal
      const int k = kkt_comp(a, s);
      const int32_t* t = a.tmpl + RT_STRIDE * k;
      const int rx = t[0], ru = t[1];
      const int cnt = a.euler ? rx + 1 + ru : 2 * (rx + ru) + a.free_tf;
      const int64_t rel = s - a.kcbase[k];
      const int64_t j = rel / (cnt + 1);
      const int e = (int)(rel - j * (cnt + 1));
      row = a.n + a.nb + (int64_t)k * a.N + j;
      if (e == cnt) col = row;
      else if (a.euler) {
        if (e < rx) col = (int64_t)a.nx * j + t[2 + e];
        else if (e == rx) col = (int64_t)a.nx * (j + 1) + k;
        else col = a.uoff + (int64_t)a.nu * j + t[2 + RT_XV + (e - rx - 1)];
      } else if (e == 2 * (rx + ru)) col = a.n - 1;
      else if (e < rx) col = (int64_t)a.nx * j + t[2 + e];
      else if (e < 2 * rx) col = (int64_t)a.nx * (j + 1) + t[2 + (e - rx)];
      else if (e < 2 * rx + ru) col = a.uoff + (int64_t)a.nu * j + t[2 + RT_XV + (e - 2 * rx)];
      else col = a.uoff + (int64_t)a.nu * (j + 1) + t[2 + RT_XV + (e - 2 * rx - ru)];
    }
    a.rows[s] = (int32_t)row;
    a.cols[s] = (int32_t)col;
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
  a.euler = P.scheme == OCP_SCHEME_EULER;
  a.kb_xn = (int64_t)a.kx * P.nun;
  a.npath = P.npath; a.nun = P.nun; a.prow0 = P.nb + (int64_t)h->nx * h->N;
  a.kpbase = h->d_pbase + (P.npath + 1); a.poff = h->d_poff; a.pv = h->d_pv;
  a.nbin = P.nbin; a.kbbase = h->d_bbase + (P.nbin + 1); a.boff = h->d_boff; a.bv = h->d_bv;
  for (int i = 0; i < a.kx; ++i) { a.ksrc[i] = (int16_t)P.kxt[i].src; a.ka[i] = (int16_t)P.kxt[i].a; a.kb[i] = (int16_t)P.kxt[i].b; }
  for (int i = 0; i < a.ku; ++i) {
    a.ksrc[KKT_TMAX + i] = (int16_t)P.kut[i].src;
    a.ka[KKT_TMAX + i] = (int16_t)P.kut[i].a;
    a.kb[KKT_TMAX + i] = (int16_t)P.kut[i].b;
  }
  if (h->nx + 5 + P.npath + P.nbin > KKT_MAXREG) return OCP_EDIM;
  auto add = [&](int kind, int64_t out, int64_t len, uint32_t period, int64_t src, uint32_t stride) {
    if (len <= 0) return;
    KRegion& r = a.reg[a.nreg++];
    r.kind = kind; r.out = out; r.len = (uint32_t)len; r.period = period; r.src = src; r.stride = stride;
  };
  add(KR_X, 0, a.kb_xn, (uint32_t)a.kx, 0, (uint32_t)P.hx);
  add(KR_XN, a.kb_xn, P.kb_u - a.kb_xn, 1, 0, 1);
  add(KR_U, P.kb_u, P.kb_t - P.kb_u, (uint32_t)a.ku, P.hbase_u, (uint32_t)P.hu);
  add(KR_TF, P.kb_t, P.kb_c - P.kb_t, 1, P.hbase_t, 1);
  add(KR_BND, P.kb_c, 2 * P.nb, 2, 0, 1);
  for (int k = 0; k < h->nx; ++k)
    add(KR_DEF, P.kcbase[k], P.kcbase[k + 1] - P.kcbase[k], (uint32_t)(P.row_count(k) + 1), P.jbase[k],
        (uint32_t)P.row_count(k));
  for (int p = 0; p < P.npath; ++p)  // path rows: the same layout (entries, then the diagonal)
    add(KR_DEF, P.kpbase[p], P.kpbase[p + 1] - P.kpbase[p], (uint32_t)(P.psupp[p].size() + 1), P.jpbase[p],
        (uint32_t)P.psupp[p].size());
  for (int q = 0; q < P.nbin; ++q)  // boundary-inequality rows: one row each (entries, then the diagonal)
    add(KR_DEF, P.kbbase[q], P.kbbase[q + 1] - P.kbbase[q], (uint32_t)(P.bsupp[q].size() + 1), P.jbbase[q],
        (uint32_t)P.bsupp[q].size());
  // blocks of the values kernel: KKT_ROWS periods of a row region per block, or
  // blockDim * KKT_ROWS slots of a short region
  uint32_t b = 0;
  for (int r = 0; r < a.nreg; ++r) {
    KRegion& R = a.reg[r];
    if (R.period > 1024) return OCP_EDIM;  // kkt_div's exactness bound
    R.block0 = b;
    const bool short_r = R.kind == KR_TF || R.kind == KR_BND || R.kind == KR_XN;
    const int64_t nb = short_r ? ((int64_t)R.len + 256 * KKT_ROWS - 1) / (256 * KKT_ROWS)
                                                              : ((int64_t)(R.len / R.period) + KKT_ROWS - 1) / KKT_ROWS;
    b += (uint32_t)nb;
  }
  a.nblocks = b;
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
  OCP_RANGE();
  if (!h || !nnzk) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  if (h->pat.nnzk < 0) return OCP_EDIM;
  *nnzk = h->pat.nnzk;
  return OCP_OK;
}

ocp_status ocp_kkt_structure(ocp_t* h, int32_t* rows, int32_t* cols, void* stream) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  if (!rows || !cols) return set_err(h, OCP_EINVAL, "rows and cols are required");
  KktArgs a;
  if (kkt_fill(h, a) != OCP_OK) return set_err(h, OCP_EDIM, "KKT matrix too large for the int32 interface");
  a.rows = rows; a.cols = cols;
  k_kkt_structure<<<kkt_grid(h, a.nnzk), 256, 0, (cudaStream_t)stream>>>(a);
  return cuda_err(h, cudaGetLastError(), "KKT structure launch");
}

ocp_status ocp_kkt_values(ocp_t* h, const double* hvals, const double* jvals, const double* sigma_x,
                          double delta_w, double delta_c, double* kvals, void* stream) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  if (!hvals || !jvals || !kvals) return set_err(h, OCP_EINVAL, "hvals, jvals and kvals are required");
  if (((uintptr_t)hvals | (uintptr_t)jvals | (uintptr_t)kvals | (uintptr_t)sigma_x) & 7u)
    return set_err(h, OCP_EINVAL, "arrays must be 8-byte aligned");
  KktArgs a;
  if (kkt_fill(h, a) != OCP_OK) return set_err(h, OCP_EDIM, "KKT matrix too large for the int32 interface");
  a.hv = hvals; a.jv = jvals; a.sx = sigma_x; a.out = kvals; a.dw = delta_w; a.dc = delta_c;
  k_kkt_values<<<a.nblocks, 256, 0, (cudaStream_t)stream>>>(a);
  return cuda_err(h, cudaGetLastError(), "KKT values launch");
}

}  // extern "C"
