// The per-variable scatter map of the Jacobian (CSC of the COO value array) and the generic
// J^T w over it.
//
// For every column c (unknown) the map lists the COO slots of J that hold an entry of that
// column, by increasing row: colptr[c] .. colptr[c+1]-1 index rows[] (the row of the entry)
// and slots[] (its position in jvals).  The pattern compiler gives, for each local variable v
// of a node, the ordered list of (component k, row side, entry position e) that reference it
// (side 1: the row of the previous interval, k's row j-1; side 0: the row of the node's own
// interval, k's row j).  A column's entries are then, in row order: its boundary row (X_{0,v}
// or a final row X_{N,v}), the defect rows from that list, the path rows of its node, and the
// boundary-inequality rows (X_0 and X_N only).  The free final time's column holds one entry
// per defect row (the last entry of each).  The map is built by one thread per column from the
// templates: a count pass, an exclusive scan, a fill pass (no sort).
//
// ocp_jtprod_coo computes J^T w from stored J values by this map: one thread per column adds
// its entries in row order; the free final time's column is one CTA's fixed-order reduction.
#include <algorithm>
#include <cstring>
#include <vector>

#include "ocp_internal.h"

namespace ocpg {

struct MapArgs {
  int32_t* cnt;          // count pass: entries per column (n)
  const int32_t* ptr;    // fill pass: column starts (n + 1)
  int32_t* rows;
  int32_t* slots;
  const int32_t* vt_off; // per local variable v: its references vt_*[vt_off[v] .. vt_off[v+1])
  const int32_t* vt_k;
  const int32_t* vt_side;
  const int32_t* vt_e;
  const int64_t* jbase;  // nx + 1
  const int32_t* fin;    // components of the final rows
  const int64_t* pbase;  // path rows: first slot of row p (npath + 1)
  const int32_t* poff;   // path supports: pv[poff[p] .. poff[p+1])
  const int32_t* pv;
  const int64_t* bbase;  // boundary-inequality rows: first slot of row q (nbin + 1)
  const int32_t* boff;   // their supports (local indices of (X_0, X_N))
  const int32_t* bv;
  int64_t N, nb, ncols, nun, uoff, prow0, brow0;   // ncols: columns handled per thread (n without tf)
  int nx, nu, nfin, npath, nbin;
};

template <bool FILL>
__global__ void __launch_bounds__(256) k_scatter_map(const __grid_constant__ MapArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < a.ncols; c += stride) {
    int64_t j;
    int v;
    if (c < a.uoff) { j = c / a.nx; v = (int)(c - j * a.nx); }
    else { const int64_t r = c - a.uoff; j = r / a.nu; v = a.nx + (int)(r - j * a.nu); }
    int32_t n = 0;
    int64_t t = FILL ? a.ptr[c] : 0;
    auto emit = [&](int64_t row, int64_t slot) {
      if (FILL) { a.rows[t] = (int32_t)row; a.slots[t] = (int32_t)slot; ++t; }
      ++n;
    };
    if (v < a.nx) {  // boundary rows: X_{0,v} is row v, X_{N,fin[i]} is row nx + i
      if (j == 0) emit(v, v);
      if (j == a.N)
        for (int i = 0; i < a.nfin; ++i)
          if (a.fin[i] == v) emit(a.nx + i, a.nx + i);
    }
    for (int r = a.vt_off[v]; r < a.vt_off[v + 1]; ++r) {  // defect rows, ascending
      const int k = a.vt_k[r];
      const int64_t jr = a.vt_side[r] ? j - 1 : j;
      if (jr < 0 || jr >= a.N) continue;
      const int64_t cntk = (a.jbase[k + 1] - a.jbase[k]) / a.N;
      emit(a.nb + (int64_t)k * a.N + jr, a.jbase[k] + jr * cntk + a.vt_e[r]);
    }
    if (j < a.nun)  // path rows of node j, ascending
      for (int p = 0; p < a.npath; ++p) {
        const int s0 = a.poff[p], s1 = a.poff[p + 1];
        for (int s = s0; s < s1; ++s)
          if (a.pv[s] == v) emit(a.prow0 + (int64_t)p * a.nun + j, a.pbase[p] + j * (s1 - s0) + (s - s0));
      }
    if (v < a.nx && (j == 0 || j == a.N)) {  // boundary inequalities on X_0 or X_N
      const int lv = (j == 0) ? v : a.nx + v;
      for (int q = 0; q < a.nbin; ++q)
        for (int s = a.boff[q]; s < a.boff[q + 1]; ++s)
          if (a.bv[s] == lv) emit(a.brow0 + q, a.bbase[q] + (s - a.boff[q]));
    }
    if (!FILL) a.cnt[c] = n;
  }
}

// The free final time's column (the last one): the last entry of every defect row, row order.
__global__ void __launch_bounds__(256) k_scatter_tf(const __grid_constant__ MapArgs a, int64_t base) {
  const int64_t total = (int64_t)a.nx * a.N, stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const int k = (int)(i / a.N);
    const int64_t jr = i - (int64_t)k * a.N;
    const int64_t cntk = (a.jbase[k + 1] - a.jbase[k]) / a.N;
    a.rows[base + i] = (int32_t)(a.nb + i);
    a.slots[base + i] = (int32_t)(a.jbase[k] + jr * cntk + cntk - 1);
  }
}

// Exclusive scan of cnt[0..n) into ptr[0..n] (ptr[n] = total): per-block sums, one block
// scanning them, then the per-element pass.
constexpr int SCAN_B = 1024;
__global__ void __launch_bounds__(SCAN_B) k_scan_blocks(const int32_t* cnt, int64_t n, int64_t* bsum) {
  __shared__ int64_t s[SCAN_B];
  const int64_t i = (int64_t)blockIdx.x * SCAN_B + threadIdx.x;
  s[threadIdx.x] = i < n ? cnt[i] : 0;
  __syncthreads();
  for (int o = SCAN_B / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = s[0];
}
__global__ void __launch_bounds__(32) k_scan_sums(int64_t* bsum, int64_t nb) {
  if (threadIdx.x != 0) return;
  int64_t acc = 0;
  for (int64_t b = 0; b < nb; ++b) { const int64_t v = bsum[b]; bsum[b] = acc; acc += v; }
  bsum[nb] = acc;
}
__global__ void __launch_bounds__(SCAN_B) k_scan_apply(const int32_t* cnt, int64_t n, const int64_t* bsum,
                                                      int64_t nb, int32_t* ptr) {
  __shared__ int64_t s[SCAN_B];
  const int64_t i = (int64_t)blockIdx.x * SCAN_B + threadIdx.x;
  const int64_t v = i < n ? cnt[i] : 0;
  s[threadIdx.x] = v;
  __syncthreads();
  for (int o = 1; o < SCAN_B; o <<= 1) {  // inclusive Hillis-Steele scan of the block
    const int64_t add = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
    __syncthreads();
    s[threadIdx.x] += add;
    __syncthreads();
  }
  if (i < n) ptr[i] = (int32_t)(bsum[blockIdx.x] + s[threadIdx.x] - v);
  if (blockIdx.x == 0 && threadIdx.x == 0) ptr[n] = (int32_t)bsum[nb];
}

// Host: per local variable, the (k, side, e) references in row order.
static void variable_templates(const Pattern& P, std::vector<int32_t>& off, std::vector<int32_t>& vk,
                               std::vector<int32_t>& side, std::vector<int32_t>& ve) {
  const bool euler = P.scheme == OCP_SCHEME_EULER;
  off.assign(1, 0);
  vk.clear(); side.clear(); ve.clear();
  auto add = [&](int k, int sd, int e) { vk.push_back(k); side.push_back(sd); ve.push_back(e); };
  for (int v = 0; v < P.nz; ++v) {
    for (int k = 0; k < P.nx; ++k) {
      const RowTemplate& T = P.rows[k];
      if (v < P.nx) {
        if (euler) {
          if (k == v) add(k, 1, T.rx);  // X_{j,k} in row (k, j-1)
          for (int e = 0; e < T.rx; ++e)
            if (T.xv[e] == v) add(k, 0, e);
        } else {
          for (int e = 0; e < T.rx; ++e)
            if (T.xv[e] == v) add(k, 1, T.rx + e);  // right node of row (k, j-1)
          for (int e = 0; e < T.rx; ++e)
            if (T.xv[e] == v) add(k, 0, e);         // left node of row (k, j)
        }
      } else {
        const int i = v - P.nx;
        if (euler) {
          for (int e = 0; e < T.ru; ++e)
            if (T.uv[e] == i) add(k, 0, T.rx + 1 + e);
        } else {
          for (int e = 0; e < T.ru; ++e)
            if (T.uv[e] == i) add(k, 1, 2 * T.rx + T.ru + e);
          for (int e = 0; e < T.ru; ++e)
            if (T.uv[e] == i) add(k, 0, 2 * T.rx + e);
        }
      }
    }
    off.push_back((int32_t)vk.size());
  }
}

// Device copies of the scatter map, built on first use and dropped when the pattern changes.
struct ScatterMap {
  int64_t n = 0, nnzj = 0;
  int32_t* ptr = nullptr;
  int32_t* rows = nullptr;
  int32_t* slots = nullptr;
};

void scatter_map_free(ocp* h) {
  if (!h || !h->smap) return;
  cudaFree(h->smap->ptr); cudaFree(h->smap->rows); cudaFree(h->smap->slots);
  delete h->smap;
  h->smap = nullptr;
}

// Writes the map into ptr (n + 1), rows and slots (nnzj) on stream s.
static ocp_status build_map(ocp* h, int32_t* ptr, int32_t* rows, int32_t* slots, cudaStream_t s) {
  const Pattern& P = h->pat;
  std::vector<int32_t> off, vk, side, ve;
  variable_templates(P, off, vk, side, ve);
  if (vk.empty()) { vk.push_back(0); side.push_back(0); ve.push_back(0); }
  const int64_t ncols = P.n - P.free_tf;
  const int64_t nblk = (P.n + SCAN_B - 1) / SCAN_B;
  // scratch: the templates, counts (n) and block sums (nblk + 1)
  const size_t tb = sizeof(int32_t) * (off.size() + 3 * vk.size());
  const size_t cb = sizeof(int32_t) * (size_t)std::max<int64_t>(P.n, 1);
  const size_t bb = sizeof(int64_t) * (size_t)(nblk + 1);
  char* scratch = nullptr;
  cudaError_t e = ocpg::dev_malloc(&scratch, tb + cb + bb + 64);
  if (e != cudaSuccess) return cuda_err(h, e, "cudaMalloc(scatter map scratch)");
  int32_t* d_off = reinterpret_cast<int32_t*>(scratch);
  int32_t* d_k = d_off + off.size();
  int32_t* d_side = d_k + vk.size();
  int32_t* d_e = d_side + vk.size();
  int32_t* d_cnt = reinterpret_cast<int32_t*>(scratch + ((tb + 15) / 16) * 16);
  int64_t* d_bsum = reinterpret_cast<int64_t*>(scratch + ((tb + 15) / 16) * 16 + ((cb + 15) / 16) * 16);
  std::vector<int32_t> host(off);
  host.insert(host.end(), vk.begin(), vk.end());
  host.insert(host.end(), side.begin(), side.end());
  host.insert(host.end(), ve.begin(), ve.end());
  e = cudaMemcpyAsync(d_off, host.data(), tb, cudaMemcpyHostToDevice, s);
  MapArgs a;
  memset(&a, 0, sizeof(a));
  a.cnt = d_cnt; a.ptr = ptr; a.rows = rows; a.slots = slots;
  a.vt_off = d_off; a.vt_k = d_k; a.vt_side = d_side; a.vt_e = d_e;
  a.jbase = h->d_jbase; a.fin = h->d_fin;
  a.pbase = h->d_pbase; a.poff = h->d_poff; a.pv = h->d_pv;
  a.bbase = h->d_bbase; a.boff = h->d_boff; a.bv = h->d_bv;
  a.N = h->N; a.nb = P.nb; a.ncols = ncols; a.nun = P.nun; a.uoff = (int64_t)h->nx * (h->N + 1);
  a.prow0 = P.nb + (int64_t)h->nx * h->N;
  a.brow0 = a.prow0 + (int64_t)P.npath * P.nun;
  a.nx = h->nx; a.nu = h->nu; a.nfin = (int)P.fin.size(); a.npath = P.npath; a.nbin = P.nbin;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((ncols + 255) / 256, (int64_t)h->num_sms * 16));
  if (e == cudaSuccess) {
    k_scatter_map<false><<<grid, 256, 0, s>>>(a);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && P.free_tf) {  // the tf column's count
    const int32_t tfc = (int32_t)((int64_t)h->nx * h->N);
    e = cudaMemcpyAsync(d_cnt + ncols, &tfc, sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // tfc lives on this stack frame
  }
  if (e == cudaSuccess) {
    k_scan_blocks<<<(unsigned)nblk, SCAN_B, 0, s>>>(d_cnt, P.n, d_bsum);
    k_scan_sums<<<1, 32, 0, s>>>(d_bsum, nblk);
    k_scan_apply<<<(unsigned)nblk, SCAN_B, 0, s>>>(d_cnt, P.n, d_bsum, nblk, ptr);
    k_scatter_map<true><<<grid, 256, 0, s>>>(a);
    if (P.free_tf) {
      const int64_t base = P.nnzj - (int64_t)h->nx * h->N;  // the last column's entries come last
      const int g2 = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)h->nx * h->N + 255) / 256, (int64_t)h->num_sms * 16));
      k_scatter_tf<<<g2, 256, 0, s>>>(a, base);
    }
    e = cudaGetLastError();
  }
  cudaError_t e2 = cudaStreamSynchronize(s);  // the scratch is released below
  if (e == cudaSuccess) e = e2;
  cudaFree(scratch);
  return e == cudaSuccess ? OCP_OK : cuda_err(h, e, "scatter map kernels");
}

static ocp_status map_ready(ocp* h, cudaStream_t s) {
  const Pattern& P = h->pat;
  if (h->smap && h->smap->n == P.n && h->smap->nnzj == P.nnzj) return OCP_OK;
  scatter_map_free(h);
  ScatterMap* m = new ScatterMap();
  h->smap = m;
  cudaError_t e = ocpg::dev_malloc(&m->ptr, sizeof(int32_t) * (size_t)(P.n + 1));
  if (e == cudaSuccess) e = ocpg::dev_malloc(&m->rows, sizeof(int32_t) * (size_t)std::max<int64_t>(P.nnzj, 1));
  if (e == cudaSuccess) e = ocpg::dev_malloc(&m->slots, sizeof(int32_t) * (size_t)std::max<int64_t>(P.nnzj, 1));
  if (e != cudaSuccess) {
    scatter_map_free(h);
    return cuda_err(h, e, "cudaMalloc(scatter map)");
  }
  ocp_status st = build_map(h, m->ptr, m->rows, m->slots, s);
  if (st != OCP_OK) { scatter_map_free(h); return st; }
  m->n = P.n; m->nnzj = P.nnzj;
  return OCP_OK;
}

// J^T w from stored values: one thread per column, entries in row order.
__global__ void __launch_bounds__(256) k_jtprod_coo(const int32_t* __restrict__ ptr, const int32_t* __restrict__ rows,
                                                    const int32_t* __restrict__ slots, const double* __restrict__ jv,
                                                    const double* __restrict__ w, double* out, int64_t ncols) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncols; c += stride) {
    double acc = 0.0;
    for (int32_t t = __ldg(ptr + c); t < __ldg(ptr + c + 1); ++t)
      acc = fma(__ldg(jv + __ldg(slots + t)), __ldg(w + __ldg(rows + t)), acc);
    out[c] = acc;
  }
}
// The free final time's column: per-thread strided sums, then a fixed tree (one CTA).
__global__ void __launch_bounds__(1024) k_jtprod_coo_long(const int32_t* __restrict__ ptr,
                                                          const int32_t* __restrict__ rows,
                                                          const int32_t* __restrict__ slots,
                                                          const double* __restrict__ jv,
                                                          const double* __restrict__ w, double* out, int64_t c) {
  __shared__ double s[1024];
  const int32_t t0 = ptr[c], t1 = ptr[c + 1];
  double acc = 0.0;
  for (int32_t t = t0 + threadIdx.x; t < t1; t += 1024) acc = fma(jv[slots[t]], w[rows[t]], acc);
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] = s[threadIdx.x] + s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = s[0];
}

}  // namespace ocpg

using namespace ocpg;

extern "C" {

ocp_status ocp_jac_scatter_map(ocp_t* h, int32_t* colptr, int32_t* rows, int32_t* slots, void* stream) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  if (!colptr || !rows || !slots) return set_err(h, OCP_EINVAL, "colptr, rows and slots are required");
  return build_map(h, colptr, rows, slots, (cudaStream_t)stream);
}

ocp_status ocp_jtprod_coo(ocp_t* h, const double* jvals, const double* w, double* Jtw, void* stream) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  if (!jvals || !w || !Jtw) return set_err(h, OCP_EINVAL, "jvals, w and Jtw are required");
  if (((uintptr_t)jvals | (uintptr_t)w | (uintptr_t)Jtw) & 7u) return set_err(h, OCP_EINVAL, "arrays must be 8-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  ocp_status st = map_ready(h, s);
  if (st != OCP_OK) return st;
  const ScatterMap* m = h->smap;
  const int64_t ncols = h->pat.n - h->pat.free_tf;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((ncols + 255) / 256, (int64_t)h->num_sms * 16));
  k_jtprod_coo<<<grid, 256, 0, s>>>(m->ptr, m->rows, m->slots, jvals, w, Jtw, ncols);
  if (h->pat.free_tf) k_jtprod_coo_long<<<1, 1024, 0, s>>>(m->ptr, m->rows, m->slots, jvals, w, Jtw, ncols);
  return cuda_err(h, cudaGetLastError(), "k_jtprod_coo launch");
}

}  // extern "C"
