// Fused FP64 evaluation kernels for models with a few states per node (one thread per node).
//
// Work decomposition.  A CTA of TILE threads evaluates TILE consecutive nodes r0..r0+TILE-1
// and OWNS the first TILE-1 of them: it writes their Hessian blocks, gradient entries and
// objective terms, and it writes the complete defect rows (k, j) for j = r0..r0+TILE-2
// (row (k, j) couples nodes j and j+1, paper Sec. 5 defect generator).  Consecutive tiles
// overlap by one node, so every slot is written exactly once by one thread, without atomics,
// at the cost of evaluating 1/TILE of the nodes twice.  CTAs are persistent and walk the
// tiles in a fixed round-robin order.
//
// Data movement.  Each thread loads its node z_j = (X_j, U_j) and, for the Hessian, the
// multiplier sums ybar_{j,k} = y_{k,j-1} + y_{k,j} (component-major, coalesced).  The tile's
// Jacobian rows are staged in shared memory in their final COO order (each component's rows
// one contiguous range) and leave by TMA bulk copies; Hessian blocks, gradient entries and the
// node-local products are stored directly by their thread; defect rows and Jv rows are
// consecutive in j and stored directly.
//
// Objective.  Each thread accumulates 2 w_j f0(z_j) = sum_a g_a d_a (g the gradient entry,
// d = z - ref) over its nodes; a fixed-shape tree reduces it per tile into the tile's slot,
// and the last CTA to finish (completion ticket) sums the slots in tile order.  The result is
// therefore deterministic for a given tile size, whatever the grid.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "model_base.cuh"
#include "ocp_internal.h"

namespace ocpg {

// Max-template of the node Hessian block: every dynamics pair plus every diagonal entry
// (the cost f0 is a diagonal quadratic), in canonical (a, b) order.  The host decides
// which diagonal entries are structural (cost weight != 0) and passes their positions.
template <class M>
struct HTmpl {
  static constexpr int CAP = M::NZ * (M::NZ + 1) / 2;
  int n = 0, nxblk = 0;
  int a[CAP] = {}, b[CAP] = {}, dyn[CAP] = {};
  bool diag[CAP] = {};
  constexpr HTmpl() {
    for (int aa = 0; aa < M::NZ; ++aa)
      for (int bb = 0; bb <= aa; ++bb) {
        int d = -1;
        for (int e = 0; e < M::NHD; ++e)
          if (M::HA(e) == aa && M::HB(e) == bb) d = e;
        if (d >= 0 || aa == bb) {
          a[n] = aa; b[n] = bb; dyn[n] = d; diag[n] = (aa == bb);
          if (aa < M::NX) ++nxblk;
          ++n;
        }
      }
  }
};

template <class M>
struct NodeArgs {
  const double* __restrict__ x;
  const double* __restrict__ y;
  const double* __restrict__ v;   // products: direction
  double* f;
  double* c;
  double* g;
  double* jv;
  double* hv;
  double* out;                    // products: result
  const double* __restrict__ wv;  // fused step: direction of J^T w (length m)
  double* ojv;                    // fused step: J v   (length m)
  double* ojtv;                   // fused step: J^T w (length n)
  double* ohv;                    // fused step: H v   (length n)
  double* partials;
  unsigned* counter;
  double* dmu;                    // jtprod: (dc/dp)^T w (M::NP doubles); hprod: the mixed term's dot
  const double* pdir_dev;         // jprod: parameter direction (device scalar) or null
  const double* mixw;             // hprod: multipliers of the mixed parameter term or null
  const double* mixs;             // hprod: scale of the mixed term (device scalar)
  double pdir;                    // jprod: parameter direction (host scalar)
  const double* p0_dev;           // model parameters read from the device (or null: K as given)
  int64_t N, nb, B, E, ntiles, uoff;  // uoff = nx (N+1): first U entry of x
  int has_final, has_ref, range;
  const double* xtrack;            // time-varying state reference, (N+1) x ntrk node-major, or null
  int ntrk;
  int8_t trk[M::NX];               // column of state k in xtrack, or -1 (constant reference)
  ModelConst K;
  double cq_in[M::NZ], cq_end[M::NZ];  // 2 sigma w q on the diagonal (interior / end node)
  double gq_in[M::NZ], gq_end[M::NZ];  // 2 w q  (gradient)
  double ref[M::NZ];
  int64_t jbase[M::NX];
  int64_t hbase_u;
  int hx, hu;
  int8_t hpos[HTmpl<M>::CAP];
};

template <class M>
__host__ __device__ constexpr int row_count(int k) { return 2 * (M::RX(k) + M::RU(k)); }
template <class M>
__host__ __device__ constexpr int jrow_total() {
  int s = 0;
  for (int k = 0; k < M::NX; ++k) s += row_count<M>(k);
  return s;
}
template <class M>
__host__ __device__ constexpr int jrow_off(int k) {
  int s = 0;
  for (int q = 0; q < k; ++q) s += row_count<M>(q);
  return s;
}

template <class M, int TILE, int NPT, unsigned OUT>
struct EvalSmem {
  static constexpr int R = NPT * TILE - 1;
  static constexpr int J = (OUT & O_J) ? jrow_total<M>() * R : 0;
  static constexpr int total = J + TILE;
  static constexpr size_t bytes = sizeof(double) * total;
};

// Sums use fma(a, one, b) with one = 1.0 read at run time (see fadd in models.cuh).
__device__ __forceinline__ double warp_sum(double v, double one) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fma(__shfl_xor_sync(0xffffffffu, v, o), one, v);
  return v;
}

// Fixed-order CTA sum; result valid in thread 0.  `red` holds TILE/32 doubles.
template <int TILE>
__device__ __forceinline__ double cta_sum(double v, double* red, double one = 1.0) {
  v = warp_sum(v, one);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < TILE / 32; ++i) s = fma(red[i], one, s);
  }
  return s;
}

// Fixed-order sum of one value per thread over the CTA through shared memory: warp 0 adds
// the TILE/32 values of each lane position, then a warp tree.  Result valid in thread 0.
// (Cheaper on the FP64 pipe than a tree in every warp.)  `red` holds TILE doubles.
template <int TILE>
__device__ __forceinline__ double tile_sum(double v, double* red, double one) {
  red[threadIdx.x] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = red[threadIdx.x];
#pragma unroll
    for (int i = 1; i < TILE / 32; ++i) s = fma(red[threadIdx.x + 32 * i], one, s);
    s = warp_sum(s, one);
  }
  return s;
}

// tile_sum of COUNT values per thread at once (the same fixed order for each), with one barrier
// for all of them.  `red` holds COUNT * TILE doubles; results valid in thread 0.
template <int TILE, int COUNT>
__device__ __forceinline__ void tile_sum_n(const double (&v)[COUNT], double* red, double one, double (&out)[COUNT]) {
#pragma unroll
  for (int q = 0; q < COUNT; ++q) red[q * TILE + threadIdx.x] = v[q];
  __syncthreads();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int q = 0; q < COUNT; ++q) {
      double s = red[q * TILE + threadIdx.x];
#pragma unroll
      for (int i = 1; i < TILE / 32; ++i) s = fma(red[q * TILE + threadIdx.x + 32 * i], one, s);
      out[q] = warp_sum(s, one);
    }
  }
}

// Completion of a reduction over tiles: every tile t stored its fixed-order CTA sum of value
// i < count in partials[i * ntiles + t]; the last CTA to finish (completion ticket) adds each
// partials[i * ntiles + 0..ntiles) in a fixed order (strided per thread, then a fixed tree)
// and writes scale * sum to dst[i].  The result depends only on the tile size, not on the grid
// or the kernel variant.
template <int TILE, int COUNT = 1>
__device__ __forceinline__ void finish_tiles(const double* partials, int64_t ntiles, unsigned* counter, double* dst,
                                             double scale, double* red) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned ticket = atomicAdd(counter, 1u);
    s_last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
#pragma unroll 1
  for (int q = 0; q < COUNT; ++q) {
    const double* part = partials + q * ntiles;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < ntiles; i += TILE) s = s + __ldcg(part + i);
    s = cta_sum<TILE>(s, red);
    if (threadIdx.x == 0) dst[q] = scale * s;
  }
  if (threadIdx.x == 0) *counter = 0u;
}

template <class M>
__device__ __forceinline__ void load_node(const NodeArgs<M>& a, int64_t j, double (&z)[M::NZ]) {
#pragma unroll
  for (int k = 0; k < M::NX; ++k) z[k] = __ldg(a.x + M::NX * j + k);
#pragma unroll
  for (int i = 0; i < M::NU; ++i) z[M::NX + i] = __ldg(a.x + a.uoff + M::NU * j + i);
}

// The model constants of a launch.  With PAR (device-resident parameters: params[0] bound by
// ocp_bind_param0, or the model's whole parameter vector for one call) the
// parameter-dependent constants are recomputed from them.  PAR is a
// template argument rather than a run-time test: a branch this short is if-converted, and
// its predicated-off FP64 instructions would still take FP64 pipe slots in every warp.
template <class M, bool PAR>
__device__ __forceinline__ ModelConst launch_consts(const NodeArgs<M>& a) {
  ModelConst K = a.K;
  if constexpr (PAR) M::device_params(K, a.p0_dev);
  return K;
}

// ybar_k = w_{k,j-1} + w_{k,j} over the defect rows of component k (zero outside 0..N-1)
template <class M>
__device__ __forceinline__ void load_bar(const NodeArgs<M>& a, const ModelConst& K, const double* w, int64_t j, double (&wb)[M::NX],
                                         double (&wl)[M::NX], double (&wr)[M::NX]) {
#pragma unroll
  for (int k = 0; k < M::NX; ++k) {
    const double* row = w + a.nb + (int64_t)k * a.N;
    wl[k] = (j >= 1) ? __ldg(row + j - 1) : 0.0;
    wr[k] = (j < a.N) ? __ldg(row + j) : 0.0;
    wb[k] = fadd(K, wl[k], wr[k]);
  }
}

// ======================================================================================
// Fused evaluation: objective, constraints, gradient, Jacobian values, Hessian values.
// ======================================================================================
template <class M>
__device__ __forceinline__ void node_cq(const NodeArgs<M>& a, bool endp, double (&cqd)[M::NZ]) {
#pragma unroll
  for (int v = 0; v < M::NZ; ++v) cqd[v] = endp ? a.cq_end[v] : a.cq_in[v];
}

template <class M>
__device__ __forceinline__ void load_ybar(const NodeArgs<M>& a, const ModelConst& K, const double* w, int64_t j,
                                          double (&wb)[M::NX]) {
#pragma unroll
  for (int k = 0; k < M::NX; ++k) {
    if (M::HK(k)) {
      const double* row = w + a.nb + (int64_t)k * a.N;
      const double wl = (j >= 1) ? __ldg(row + j - 1) : 0.0;
      const double wr = (j < a.N) ? __ldg(row + j) : 0.0;
      wb[k] = fadd(K, wl, wr);
    } else {
      wb[k] = 0.0;
    }
  }
}

// gradient entries g_v = 2 w_j q_v (z_v - ref_v); returns 2 w_j f0(z_j) = sum_v g_v (z_v - ref_v)
// (ref_v of a tracked state component is read from the per-node table xtrack)
template <class M, bool REF, bool WG>
__device__ __forceinline__ double node_grad(const NodeArgs<M>& a, const ModelConst& K, const double (&z)[M::NZ], bool endp,
                                           int64_t j) {
  double s = 0.0;
#pragma unroll
  for (int v = 0; v < M::NZ; ++v) {
    double rv = a.ref[v];
    if (REF && v < M::NX && a.xtrack && a.trk[v < M::NX ? v : 0] >= 0)
      rv = __ldg(a.xtrack + (int64_t)a.ntrk * j + a.trk[v < M::NX ? v : 0]);
    const double d = REF ? fsub(K, z[v], rv) : z[v];
    const double gv = fmul(K, endp ? a.gq_end[v] : a.gq_in[v], d);
    if (WG) {
      if (v < M::NX) a.g[(int64_t)M::NX * j + v] = gv;
      else a.g[a.uoff + (int64_t)M::NU * j + (v - M::NX)] = gv;
    }
    s = (v == 0) ? fmul(K, gv, d) : fma(gv, d, s);
  }
  return s;
}

// ---- per-node product terms, shared by the product kernels and the fused step -----------
// Jv: with p_k = -hh grad f_k(z_j) . v_{z_j} (+ -hh df_k/dmu * pdir), A_k = p_k + v_{X_j,k} is the
// node's share of row (k, j-1) and B_k = p_k - v_{X_j,k} its share of row (k, j); the last term
// of p_k is fused into both.
template <class M, bool PDIR>
__device__ __forceinline__ void jv_node(const ModelConst& K, const double (&mjx)[M::NX][M::MAXRX],
                                        const double (&mju)[M::NX][M::MAXRU],
                                        const double (&mdp)[M::NX], double pd, const double (&vz)[M::NZ],
                                        double (&A)[M::NX], double (&Bm)[M::NX]) {
  constexpr int NX = M::NX;
#pragma unroll
  for (int k = 0; k < NX; ++k) {
    double cf[M::MAXRX + M::MAXRU + 1], vv[M::MAXRX + M::MAXRU + 1];
    int nt = 0;
#pragma unroll
    for (int e = 0; e < M::MAXRX; ++e)
      if (e < M::RX(k) && !M::JZ(k, e)) { cf[nt] = mjx[k][e]; vv[nt] = vz[M::XV(k, e)]; ++nt; }
#pragma unroll
    for (int e = 0; e < M::MAXRU; ++e)
      if (e < M::RU(k)) { cf[nt] = mju[k][e]; vv[nt] = vz[NX + M::UV(k, e)]; ++nt; }
    if (PDIR) { cf[nt] = mdp[k]; vv[nt] = pd; ++nt; }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i + 1 < nt; ++i) s = (i == 0) ? fmul(K, cf[i], vv[i]) : fma(cf[i], vv[i], s);
    const double vk = vz[k];
    if (nt == 0) {
      A[k] = vk;
      Bm[k] = -vk;
    } else if (nt == 1) {
      A[k] = fma(cf[0], vv[0], vk);
      Bm[k] = fma(cf[0], vv[0], -vk);
    } else {
      // p = sum of all terms, then p + v and p - v (one operation fewer than fusing the last term twice)
      const double pk = fma(cf[nt - 1], vv[nt - 1], s);
      A[k] = fadd(K, pk, vk);
      Bm[k] = fsub(K, pk, vk);
    }
  }
}

// J^T w at node j: (w_{a,j-1} - w_{a,j}) + sum_k wbar_k mjx_{k,a}, the control entries
// sum_k wbar_k mju_{k,i}, plus the boundary rows' w at j = 0 / N (bnd: this CTA may hold them).
template <class M>
__device__ __forceinline__ void jtv_node(const NodeArgs<M>& a, const ModelConst& K, const double* w, int64_t j, bool bnd,
                                         const double (&mjx)[M::NX][M::MAXRX], const double (&mju)[M::NX][M::MAXRU],
                                         const double (&wl)[M::NX], const double (&wr)[M::NX],
                                         const double (&wb)[M::NX], double (&o)[M::NZ]) {
  constexpr int NX = M::NX;
  // every state entry accumulates its terms in increasing k (one pass over the row templates)
#pragma unroll
  for (int v = 0; v < NX; ++v) o[v] = fsub(K, wl[v], wr[v]);
#pragma unroll
  for (int k = 0; k < NX; ++k)
#pragma unroll
    for (int e = 0; e < M::MAXRX; ++e)
      if (e < M::RX(k) && !M::JZ(k, e)) o[M::XV(k, e)] = fma(wb[k], mjx[k][e], o[M::XV(k, e)]);
  if (bnd) {  // only CTAs holding node 0 or node N (uniform branch)
#pragma unroll
    for (int v = 0; v < NX; ++v) {
      if (j == 0) o[v] = fadd(K, o[v], __ldg(w + v));
      if (a.has_final && j == a.N) o[v] = fadd(K, o[v], __ldg(w + NX + v));
    }
  }
#pragma unroll
  for (int i = 0; i < M::NU; ++i) {
    double s = 0.0;
    bool first = true;
#pragma unroll
    for (int k = 0; k < NX; ++k)
#pragma unroll
      for (int e = 0; e < M::MAXRU; ++e)
        if (e < M::RU(k) && M::UV(k, e) == i) { s = first ? fmul(K, wb[k], mju[k][e]) : fma(wb[k], mju[k][e], s); first = false; }
    o[NX + i] = s;
  }
}

// H v at node j: the full symmetric block (structural entries only) times v_{z_j}.
template <class M>
__device__ __forceinline__ void hv_node(const NodeArgs<M>& a, const ModelConst& K, const double* hd, const double (&cqd)[M::NZ],
                                        const double (&vz)[M::NZ], double (&o)[M::NZ]) {
  constexpr HTmpl<M> HT{};
  bool first[M::NZ];
#pragma unroll
  for (int v = 0; v < M::NZ; ++v) { o[v] = 0.0; first[v] = true; }
#pragma unroll
  for (int e = 0; e < HT.n; ++e) {
    if (a.hpos[e] >= 0) {
      const int aa = HT.a[e], bb = HT.b[e];
      const double val = (HT.dyn[e] >= 0) ? hd[HT.dyn[e] >= 0 ? HT.dyn[e] : 0] : cqd[aa];
      o[aa] = first[aa] ? fmul(K, val, vz[bb]) : fma(val, vz[bb], o[aa]);
      first[aa] = false;
      if (aa != bb) {
        o[bb] = first[bb] ? fmul(K, val, vz[aa]) : fma(val, vz[aa], o[bb]);
        first[bb] = false;
      }
    }
  }
}

template <class M>
__device__ __forceinline__ void load_vz(const NodeArgs<M>& a, const double* v, int64_t j, double (&vz)[M::NZ]) {
#pragma unroll
  for (int k = 0; k < M::NX; ++k) vz[k] = __ldg(v + M::NX * j + k);
#pragma unroll
  for (int i = 0; i < M::NU; ++i) vz[M::NX + i] = __ldg(v + a.uoff + M::NU * j + i);
}

template <class M>
__device__ __forceinline__ void store_nz(const NodeArgs<M>& a, double* out, int64_t j, const double (&o)[M::NZ]) {
#pragma unroll
  for (int v = 0; v < M::NX; ++v) out[M::NX * j + v] = o[v];
#pragma unroll
  for (int i = 0; i < M::NU; ++i) out[a.uoff + M::NU * j + i] = o[M::NX + i];
}

// One tile of the fused evaluation.  The CTA's TILE threads cover NPT*TILE consecutive
// nodes r0.. (thread t takes nodes r0 + NPT t + q, q < NPT: consecutive pairs give each thread
// independent FP64 dependency chains) and own the first NPT*TILE - 1 of them.  `a` may live in
// parameter or shared memory.  The tile's objective term (2 w_j f0 summed in a fixed order)
// goes to *partial.
template <class M, int TILE, int NPT, unsigned OUT>
__device__ __forceinline__ void node_eval_tile(const NodeArgs<M>& a, const ModelConst& K, int64_t tile, double* sm,
                                               double* sEdge, double* partial) {
  constexpr int NX = M::NX, NZ = M::NZ;
  constexpr int NT = NPT * TILE;  // nodes per tile
  constexpr bool WF = OUT & O_F, WC = OUT & O_C, WG = OUT & O_G, WJ = OUT & O_J, WH = OUT & O_H;
  constexpr bool WJV = OUT & O_JV, WJTV = OUT & O_JTV, WHV = OUT & O_HV;  // fused step products
  constexpr bool NEEDJ = WJ || WJV || WJTV, NEEDH = WH || WHV;
  // the full kernel also serves output subsets: NULL outputs are computed but not stored
  const bool sF = WF && a.f, sC = WC && a.c, sG = WG && a.g, sJ = WJ && a.jv, sH = WH && a.hv;
  constexpr HTmpl<M> HT{};
  constexpr int NHD = (M::NHD > 0) ? M::NHD : 1;
  constexpr int R = NT - 1;            // owned rows / nodes per tile
  constexpr int oRED = (OUT & O_J) ? jrow_total<M>() * R : 0;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;

  const int64_t r0 = a.B + tile * R;
  const int64_t own_end = min(r0 + R, a.E);
  const int64_t row_end = min(own_end, a.N);
  const int64_t eval_end = row_end + 1;
  const int nown = (int)(own_end - r0);
  const int nrows = (int)max(row_end - r0, (int64_t)0);
  double objterm = 0.0;
  double pa[NPT][NX], pb[NPT][NX];
  double jA[NPT][NX], jB[NPT][NX];     // fused step: node shares of the Jv rows
  const bool bnd = (r0 == 0) || (r0 + R > a.N);  // tile may hold node 0 or node N (uniform)

#pragma unroll
  for (int q = 0; q < NPT; ++q) {
    const int lt = NPT * t + q;       // node index within the tile
    const int64_t j = r0 + lt;
    const bool act = j < eval_end;
    const bool own = lt < nown;
    const bool endp = (j == 0) || (j == a.N);
    double z[NZ], yb[NX], cqd[NZ], mjx[NX][M::MAXRX], mju[NX][M::MAXRU], hd[NHD];
#pragma unroll
    for (int k = 0; k < NX; ++k) { pa[q][k] = 0.0; pb[q][k] = 0.0; jA[q][k] = 0.0; jB[q][k] = 0.0; }
    double vz[NZ];
    if (act) {
      load_node<M>(a, j, z);
      if (NEEDH) {
        load_ybar<M>(a, K, a.y, j, yb);
        node_cq<M>(a, endp, cqd);
      }
      M::template eval<WC, NEEDJ, NEEDH>(K, z, yb, cqd, pa[q], pb[q], mjx, mju, hd);
      if (WJV || WHV) load_vz<M>(a, a.v, j, vz);
      if (WJV) {
        double mdp[NX];
        jv_node<M, false>(K, mjx, mju, mdp, 0.0, vz, jA[q], jB[q]);
      }
    }
    // ---- Jacobian rows staged in shared memory: left part of row lt, right part of row lt-1
    if (WJ && act) {
#pragma unroll
      for (int k = 0; k < NX; ++k) {
        const int cnt = row_count<M>(k);
        double* sj = sm + jrow_off<M>(k) * R;
        if (lt < nrows) {
          double* rp = sj + lt * cnt;
#pragma unroll
          for (int e = 0; e < M::MAXRX; ++e)
            if (e < M::RX(k)) rp[e] = (M::XV(k, e) == k) ? (M::JZ(k, e) ? -1.0 : fma(mjx[k][e], K.one, -1.0)) : mjx[k][e];
#pragma unroll
          for (int e = 0; e < M::MAXRU; ++e)
            if (e < M::RU(k)) rp[2 * M::RX(k) + e] = mju[k][e];
        }
        if (lt >= 1 && lt - 1 < nrows) {
          double* rp = sj + (lt - 1) * cnt;
#pragma unroll
          for (int e = 0; e < M::MAXRX; ++e)
            if (e < M::RX(k)) rp[M::RX(k) + e] = (M::XV(k, e) == k) ? (M::JZ(k, e) ? 1.0 : fma(mjx[k][e], K.one, 1.0)) : mjx[k][e];
#pragma unroll
          for (int e = 0; e < M::MAXRU; ++e)
            if (e < M::RU(k)) rp[2 * M::RX(k) + M::RU(k) + e] = mju[k][e];
        }
      }
    }
    if (own) {
      if (WJTV) {
        double wb[NX], wl[NX], wr[NX], o[NZ];
        load_bar<M>(a, K, a.wv, j, wb, wl, wr);
        jtv_node<M>(a, K, a.wv, j, bnd, mjx, mju, wl, wr, wb, o);
        store_nz<M>(a, a.ojtv, j, o);
      }
      if (WHV) {
        double o[NZ];
        hv_node<M>(a, K, hd, cqd, vz, o);
        store_nz<M>(a, a.ohv, j, o);
      }
      if (WJV && bnd) {
        if (j == 0) {
#pragma unroll
          for (int k = 0; k < NX; ++k) a.ojv[k] = vz[k];
        }
        if (a.has_final && j == a.N) {
#pragma unroll
          for (int k = 0; k < NX; ++k) a.ojv[NX + k] = vz[k];
        }
      }
    }
    if (own) {
      // ---- Hessian block of node j (stored directly; X block then U block)
      if (sH) {
#pragma unroll
        for (int e = 0; e < HT.n; ++e) {
          const int p = a.hpos[e];
          if (p >= 0) {
            const double val = (HT.dyn[e] >= 0) ? hd[HT.dyn[e] >= 0 ? HT.dyn[e] : 0] : cqd[HT.a[e]];
            if (HT.a[e] < NX) a.hv[j * a.hx + p] = val;
            else a.hv[a.hbase_u + j * a.hu + p] = val;
          }
        }
      }
      // ---- gradient and objective term
      if (sG || sF) {
        double s2;
        if (a.has_ref) s2 = sG ? node_grad<M, true, true>(a, K, z, endp, j) : node_grad<M, true, false>(a, K, z, endp, j);
        else s2 = sG ? node_grad<M, false, true>(a, K, z, endp, j) : node_grad<M, false, false>(a, K, z, endp, j);
        objterm = (q == 0) ? s2 : fadd(K, objterm, s2);
      }
      // ---- boundary rows X_{0,k} (and X_{N,k}): constraint value and the constant Jacobian entry
      if (j == 0) {
#pragma unroll
        for (int k = 0; k < NX; ++k) {
          if (sC) a.c[k] = z[k];
          if (sJ) a.jv[k] = 1.0;
        }
      }
      if (a.has_final && j == a.N) {
#pragma unroll
        for (int k = 0; k < NX; ++k) {
          if (sC) a.c[NX + k] = z[k];
          if (sJ) a.jv[NX + k] = 1.0;
        }
      }
    }
  }
  // ---- defects (and Jv rows): the right node's share is this thread's next node, or lane+1's first
  double nbv[NX], nbA[NX];
  if (WC) {
#pragma unroll
    for (int k = 0; k < NX; ++k) {
      nbv[k] = __shfl_down_sync(0xffffffffu, pb[0][k], 1);
      if (lane == 0) sEdge[warp * NX + k] = pb[0][k];
    }
  }
  if (WJV) {
    constexpr int EO = (TILE / 32 + 1) * NX;
#pragma unroll
    for (int k = 0; k < NX; ++k) {
      nbA[k] = __shfl_down_sync(0xffffffffu, jA[0][k], 1);
      if (lane == 0) sEdge[EO + warp * NX + k] = jA[0][k];
    }
  }
  // the staged Jacobian rows are read by the TMA engine (async proxy) after the barrier
  if (WJ) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (WC || WJ || WJV) __syncthreads();
  if (WJV) {
    constexpr int EO = (TILE / 32 + 1) * NX;
#pragma unroll
    for (int q = 0; q < NPT; ++q) {
      const int lt = NPT * t + q;
      if (lt < nrows) {
#pragma unroll
        for (int k = 0; k < NX; ++k) {
          double right;
          if (q + 1 < NPT) right = jA[q + 1 < NPT ? q + 1 : 0][k];
          else right = (lane == 31) ? sEdge[EO + (warp + 1) * NX + k] : nbA[k];
          a.ojv[a.nb + (int64_t)k * a.N + r0 + lt] = fadd(K, jB[q][k], right);
        }
      }
    }
  }
  if (sC) {
#pragma unroll
    for (int q = 0; q < NPT; ++q) {
      const int lt = NPT * t + q;
      if (lt < nrows) {
#pragma unroll
        for (int k = 0; k < NX; ++k) {
          double right;
          if (q + 1 < NPT) right = pb[q + 1 < NPT ? q + 1 : 0][k];
          else right = (lane == 31) ? sEdge[(warp + 1) * NX + k] : nbv[k];
          a.c[a.nb + (int64_t)k * a.N + r0 + lt] = fsub(K, right, pa[q][k]);
        }
      }
    }
  }
  // ---- copy-out of the staged Jacobian rows: the tile's rows of component k are one
  // contiguous range in shared memory and in jvals.  A range whose two ends are 16-byte
  // aligned with a multiple of 16 bytes goes out as one bulk copy by the TMA engine (issued
  // by thread 0); any other range is copied by all threads, coalesced.
  if (sJ) {
    bool bulk = false;
#pragma unroll
    for (int k = 0; k < NX; ++k) {
      const int cnt = row_count<M>(k);
      const double* src = sm + jrow_off<M>(k) * R;
      double* dst = a.jv + a.jbase[k] + r0 * cnt;
      const int total = nrows * cnt;
      const unsigned bytes = 8u * (unsigned)total;
      const bool aligned = total > 0 && ((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src) | bytes) & 15u) == 0;
      if (aligned) {
        if (t == 0) {
          const unsigned saddr = static_cast<unsigned>(__cvta_generic_to_shared(src));
          asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                       :: "l"(dst), "r"(saddr), "r"(bytes) : "memory");
        }
        bulk = true;
      } else {
        for (int i = t; i < total; i += TILE) dst[i] = src[i];
      }
    }
    // the staged rows must have been read before the shared memory is reused or released
    if (bulk && t == 0) {
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    }
  }
  if (sF) {
    const double ts = tile_sum<TILE>(objterm, sm + oRED, K.one);
    if (t == 0) *partial = ts;
  }
  if (WC || WJ || WF || WJV) __syncthreads();
}

// The fused evaluation kernel.  A model may ask for a minimum of resident CTAs per SM
// (M::EVAL_MIN_CTAS > 0, a register cap for models whose fused kernels would otherwise need
// all 255 registers); by default the register allocator's own heuristic applies.
template <class M, int TILE, int NPT, unsigned OUT, bool PAR>
__device__ __forceinline__ void node_eval_kernel_body(const NodeArgs<M>& a) {
  constexpr bool WF = OUT & O_F;
  extern __shared__ __align__(16) double sm[];
  __shared__ double sEdge[2 * (TILE / 32 + 1) * M::NX];
  const ModelConst K = launch_consts<M, PAR>(a);
  for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x)
    node_eval_tile<M, TILE, NPT, OUT>(a, K, tile, sm, sEdge, a.partials + tile);
  if (WF && a.f) finish_tiles<TILE>(a.partials, a.ntiles, a.counter, a.f, 0.5, sm);
}

template <class M, int TILE, int NPT, unsigned OUT, bool PAR>
__global__ void __launch_bounds__(TILE) k_node_eval(const __grid_constant__ NodeArgs<M> a) {
  node_eval_kernel_body<M, TILE, NPT, OUT, PAR>(a);
}

template <class M, int TILE, int NPT, unsigned OUT, bool PAR>
__global__ void __launch_bounds__(TILE, (M::EVAL_MIN_CTAS > 0 ? M::EVAL_MIN_CTAS : 1))
    k_node_eval_capped(const __grid_constant__ NodeArgs<M> a) {
  node_eval_kernel_body<M, TILE, NPT, OUT, PAR>(a);
}

template <class M, int TILE, int NPT, unsigned OUT, bool PAR>
auto eval_kernel() {
  if constexpr (M::EVAL_MIN_CTAS > 0) return k_node_eval_capped<M, TILE, NPT, OUT, PAR>;
  else return k_node_eval<M, TILE, NPT, OUT, PAR>;
}

// ======================================================================================
// Jv.  Row (k,j) = (p_k(j) - v_{X_j,k}) + (p_k(j+1) + v_{X_{j+1},k}),  (B(j) + A(j+1)),
// p_k(j) = -hh grad f_k(z_j) . v_{z_j}  (+ -hh df_k/dmu(z_j) * pdir for the parameter).
// Same overlapping tiles as the evaluation; the right-node term comes from lane+1.
// ======================================================================================
template <class M, int TILE, bool PDIR, bool PAR>
__global__ void __launch_bounds__(TILE) k_node_jprod(const __grid_constant__ NodeArgs<M> a) {
  constexpr int NX = M::NX, NZ = M::NZ;
  constexpr int NHD = (M::NHD > 0) ? M::NHD : 1;
  __shared__ double sEdge[(TILE / 32 + 1) * NX];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  ModelConst K = launch_consts<M, PAR>(a);
  double pd = 0.0;
  if (PDIR) pd = a.pdir_dev ? __ldg(a.pdir_dev) : a.pdir;
  for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * (TILE - 1);
    const int64_t own_end = min(r0 + TILE - 1, a.N + 1);
    const int64_t row_end = min(own_end, a.N);
    const int nrows = (int)max(row_end - r0, (int64_t)0);
    const int64_t j = r0 + t;
    const bool act = j <= row_end;
    double p[NX], vx[NX], A[NX];
#pragma unroll
    for (int k = 0; k < NX; ++k) { p[k] = 0.0; vx[k] = 0.0; A[k] = 0.0; }
    if (act) {
      double z[NZ], vz[NZ], yb[NX], cqd[NZ], pa[NX], pb[NX], mjx[NX][M::MAXRX], mju[NX][M::MAXRU], hd[NHD];
      load_node<M>(a, j, z);
      load_vz<M>(a, a.v, j, vz);
#pragma unroll
      for (int k = 0; k < NX; ++k) vx[k] = vz[k];
      M::template eval<false, true, false>(K, z, yb, cqd, pa, pb, mjx, mju, hd);
      double mdp[NX];
      if (PDIR) M::dparam(K, z, mdp);
      jv_node<M, PDIR>(K, mjx, mju, mdp, pd, vz, A, p);
      if (j == 0) {
#pragma unroll
        for (int k = 0; k < NX; ++k) a.out[k] = vx[k];
      }
      if (a.has_final && j == a.N && t < (int)(own_end - r0)) {
#pragma unroll
        for (int k = 0; k < NX; ++k) a.out[NX + k] = vx[k];
      }
    }
    double nbv[NX];
#pragma unroll
    for (int k = 0; k < NX; ++k) {
      nbv[k] = __shfl_down_sync(0xffffffffu, A[k], 1);
      if (lane == 0) sEdge[warp * NX + k] = A[k];
    }
    __syncthreads();
    if (t < nrows) {
#pragma unroll
      for (int k = 0; k < NX; ++k) {
        const double right = (lane == 31) ? sEdge[(warp + 1) * NX + k] : nbv[k];
        a.out[a.nb + (int64_t)k * a.N + j] = fadd(K, p[k], right);
      }
    }
    __syncthreads();
  }
}

// ======================================================================================
// J^T w, node-local:  (J^T w)_{X_j,a} = (w_{a,j-1} - w_{a,j}) + sum_k wbar_k mjx_k,a(z_j)
//                     (+ w of the boundary rows at j = 0 / N);  (J^T w)_{U_j,i} likewise.
// With DPAR, also (dc/dp_i)^T w = sum_j sum_k wbar_k mdp_k,i(z_j) for every dynamics
// parameter i < M::NP (mdp = -hh df/dp; one deterministic reduction per parameter).
// ======================================================================================
template <class M, int TILE, bool DPAR, bool PAR>
__global__ void __launch_bounds__(TILE) k_node_jtprod(const __grid_constant__ NodeArgs<M> a) {
  constexpr int NX = M::NX, NZ = M::NZ;
  constexpr int NHD = (M::NHD > 0) ? M::NHD : 1;
  constexpr int NP = M::NP, NPA = (NP > 0) ? NP : 1;
  __shared__ double red[TILE * NPA];
  ModelConst K = launch_consts<M, PAR>(a);
  const int64_t nchunks = (a.E - a.B + TILE - 1) / TILE;   // the nodes [B, E) in chunks of TILE
  for (int64_t chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
    const int64_t j0 = a.B + chunk * TILE, j = j0 + threadIdx.x;
    const bool bnd = (j0 == 0) || (j0 + TILE > a.N);  // chunk may hold node 0 or node N (uniform)
    double acc[NPA];
#pragma unroll
    for (int i = 0; i < NPA; ++i) acc[i] = 0.0;
    if (j < a.E) {
      double z[NZ], yb[NX], cqd[NZ], pa[NX], pb[NX], mjx[NX][M::MAXRX], mju[NX][M::MAXRU], hd[NHD];
      double wb[NX], wl[NX], wr[NX];
      load_node<M>(a, j, z);
      load_bar<M>(a, K, a.v, j, wb, wl, wr);
      double mdp[NX][NPA];
      if constexpr (DPAR && M::FUSED_DP) {   // J and -hh df/dp from one set of intermediates
        M::template eval<false, true, false, true>(K, z, yb, cqd, pa, pb, mjx, mju, hd, mdp);
      } else {
        M::template eval<false, true, false>(K, z, yb, cqd, pa, pb, mjx, mju, hd);
        if constexpr (DPAR && NP > 0 && !M::FUSED_DP) M::dparams(K, z, mdp);
      }
      double o[NZ];
      jtv_node<M>(a, K, a.v, j, bnd, mjx, mju, wl, wr, wb, o);
      store_nz<M>(a, a.out, j, o);
      if (DPAR && NP > 0) {
#pragma unroll
        for (int i = 0; i < NPA; ++i)
#pragma unroll
          for (int k = 0; k < NX; ++k)
            if (M::DP(k, i)) acc[i] = fma(wb[k], mdp[k][i], acc[i]);
      }
    }
    if (DPAR) {
      double ts[NPA];
      tile_sum_n<TILE, NPA>(acc, red, K.one, ts);
      if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NPA; ++i) a.partials[i * nchunks + chunk] = ts[i];
      }
      __syncthreads();
    }
  }
  if (DPAR) finish_tiles<TILE, NPA>(a.partials, nchunks, a.counter, a.dmu, 1.0, red);
}

// ======================================================================================
// H v, node-local: the full symmetric block of node j times v_{z_j}.
// With MIX (autograd double backward), also adds mixs * m_j, m_j = sum_k mixwbar_k
// (-hh d2 f_k / dmu dz)(z_j), and reduces sum_j m_j . v_{z_j} into *dmu.
// ======================================================================================
template <class M, int TILE, bool MIX, bool PAR>
__global__ void __launch_bounds__(TILE) k_node_hprod(const __grid_constant__ NodeArgs<M> a) {
  constexpr int NX = M::NX, NZ = M::NZ;
  constexpr int NHD = (M::NHD > 0) ? M::NHD : 1;
  constexpr HTmpl<M> HT{};
  __shared__ double red[TILE];
  ModelConst K = launch_consts<M, PAR>(a);
  double ms = 0.0;
  if (MIX) ms = a.mixs ? __ldg(a.mixs) : 0.0;
  const int64_t nchunks = (a.N + TILE) / TILE;
  for (int64_t chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
    const int64_t j = chunk * TILE + threadIdx.x;
    double acc_mu = 0.0;
    if (j <= a.N) {
      double z[NZ], vz[NZ], yb[NX], cqd[NZ], pa[NX], pb[NX], mjx[NX][M::MAXRX], mju[NX][M::MAXRU], hd[NHD];
      load_node<M>(a, j, z);
      load_ybar<M>(a, K, a.y, j, yb);
      const bool endp = (j == 0) || (j == a.N);
      node_cq<M>(a, endp, cqd);
#pragma unroll
      for (int k = 0; k < NX; ++k) vz[k] = __ldg(a.v + NX * j + k);
#pragma unroll
      for (int i = 0; i < M::NU; ++i) vz[NX + i] = __ldg(a.v + a.uoff + M::NU * j + i);
      M::template eval<false, false, true>(K, z, yb, cqd, pa, pb, mjx, mju, hd);
      double o[NZ];
      hv_node<M>(a, K, hd, cqd, vz, o);
      if (MIX) {
        double mb[NX], mg[NZ], wl[NX], wr[NX];
        load_bar<M>(a, K, a.mixw, j, mb, wl, wr);
        M::dparam_grad(K, z, mb, mg);
#pragma unroll
        for (int v = 0; v < NZ; ++v) {
          o[v] = fma(mg[v], ms, o[v]);
          acc_mu = fma(mg[v], vz[v], acc_mu);
        }
      }
      store_nz<M>(a, a.out, j, o);
    }
    if (MIX && a.dmu) {
      const double ts = tile_sum<TILE>(acc_mu, red, K.one);
      if (threadIdx.x == 0) a.partials[chunk] = ts;
      __syncthreads();
    }
  }
  if (MIX && a.dmu) finish_tiles<TILE>(a.partials, nchunks, a.counter, a.dmu, 1.0, red);
}

// ======================================================================================
// Host side
// ======================================================================================
template <class M>
void fill_args(const ocp* h, double sigma, NodeArgs<M>& a) {
  memset(&a, 0, sizeof(a));
  const Pattern& P = h->pat;
  a.N = h->N;
  a.nb = P.nb;
  a.uoff = (int64_t)M::NX * (h->N + 1);
  a.has_final = h->has_final ? 1 : 0;
  a.has_ref = h->has_ref ? 1 : 0;
  M::host_consts(h->params.data(), h->hh, a.K);
  for (int v = 0; v < M::NZ; ++v) {
    const double w = v < M::NX ? h->q[v] : h->r[v - M::NX];
    a.gq_in[v] = 2.0 * h->h * w;
    a.gq_end[v] = h->h * w;
    a.cq_in[v] = sigma * (2.0 * h->h * w);
    a.cq_end[v] = sigma * (h->h * w);
    a.ref[v] = v < M::NX ? h->xref[v] : h->uref[v - M::NX];
  }
  for (int k = 0; k < M::NX; ++k) a.jbase[k] = P.jbase[k];
  a.hbase_u = P.hbase_u;
  a.hx = P.hx;
  a.hu = P.hu;
  for (int e = 0; e < HTmpl<M>::CAP; ++e) a.hpos[e] = e < (int)P.hpos.size() ? P.hpos[e] : (int8_t)-1;
  a.partials = h->d_partials;
  a.counter = h->d_counter;
  a.p0_dev = h->p0_dev;
  a.xtrack = h->d_xtrack;
  a.ntrk = h->ntrk;
  for (int k = 0; k < M::NX; ++k) a.trk[k] = -1;
  for (int i = 0; i < h->ntrk; ++i) a.trk[h->trk_comp[i]] = (int8_t)i;
}

template <class M, int TILE, int NPT, unsigned OUT, bool PAR>
ocp_status launch_eval_k(ocp* h, const EvalCall& c, cudaStream_t s) {
  NodeArgs<M> a;
  fill_args<M>(h, c.sigma, a);
  a.x = c.x; a.y = c.y; a.f = c.f; a.c = c.c; a.g = c.g; a.jv = c.jv; a.hv = c.hv;
  a.v = c.vn; a.wv = c.vm; a.ojv = c.ojv; a.ojtv = c.ojtv; a.ohv = c.ohv;
  a.B = c.B; a.E = c.E;
  a.range = c.range ? 1 : 0;
  const int64_t nodes = c.E - c.B;
  constexpr int R = NPT * TILE - 1;
  a.ntiles = (nodes + R - 1) / R;
  if (a.ntiles < 1) a.ntiles = 1;
  if (a.ntiles > h->max_partials) return set_err(h, OCP_EDIM, "too many tiles for the reduction scratch");
  using S = EvalSmem<M, TILE, NPT, OUT>;
  auto kern = eval_kernel<M, TILE, NPT, OUT, PAR>();
  static unsigned attr_done = 0;
  if (!(attr_done & (1u << (h->device & 31)))) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::bytes);
    if (e != cudaSuccess) return cuda_err(h, e, "cudaFuncSetAttribute(eval)");
    attr_done |= 1u << (h->device & 31);
  }
  const int grid = occupancy_grid(h, (const void*)kern, TILE, S::bytes, a.ntiles);
  kern<<<grid, TILE, S::bytes, s>>>(a);
  return cuda_err(h, cudaGetLastError(), "k_node_eval launch");
}

template <class M, int TILE, int NPT, unsigned OUT>
ocp_status launch_eval_t(ocp* h, const EvalCall& c, cudaStream_t s) {
  // device parameters: every output for the Van der Pol mu (the differentiation form's bound
  // parameter); the constraints alone for the other models
  if constexpr (M::HAS_DPARAM || (M::NP > 0 && OUT == O_C)) {
    if (h->p0_dev) return launch_eval_k<M, TILE, NPT, OUT, true>(h, c, s);
  } else {
    if (h->p0_dev) return set_err(h, OCP_EMODEL, "device parameters are not provided for this output set");
  }
  return launch_eval_k<M, TILE, NPT, OUT, false>(h, c, s);
}

// ======================================================================================
// Forward Euler scheme (paper Sec. 3): defect (k, j) = X_{j+1,k} - X_{j,k} - h f_k(z_j) for
// j < N, cost sum_{j<N} h f0(z_j), controls U_0..U_{N-1}.  A row uses only its own node's f,
// so one thread per node evaluates its rows completely (tiles of TILE nodes do not overlap);
// node N contributes only X_N (identity entries, boundary rows).  The model runs with
// K.hh = h, so pa = x + h f, mjx = -h df/dx and hd = -h sum_k y_{k,j} d2f_k + sigma h d2f0.
// Row (k, j) lists the entries on X_j (the template, identity merged), X_{j+1,k}, then U_j.
// (An identity-only entry, df_k/dx_k identically zero, is the constant -1 or +1 in every kernel.)
// ======================================================================================
template <class M>
__host__ __device__ constexpr int euler_count(int k) { return M::RX(k) + 1 + M::RU(k); }
template <class M>
__host__ __device__ constexpr int euler_total() {
  int s = 0;
  for (int k = 0; k < M::NX; ++k) s += euler_count<M>(k);
  return s;
}
template <class M>
__host__ __device__ constexpr int euler_off(int k) {
  int s = 0;
  for (int q = 0; q < k; ++q) s += euler_count<M>(q);
  return s;
}

template <class M, int TILE, unsigned OUT, bool PAR>
__global__ void __launch_bounds__(TILE) k_euler(const __grid_constant__ NodeArgs<M> a) {
  constexpr int NX = M::NX, NZ = M::NZ;
  constexpr bool WF = OUT & O_F, WC = OUT & O_C, WG = OUT & O_G, WJ = OUT & O_J, WH = OUT & O_H;
  constexpr bool WJV = OUT & O_JV, WJTV = OUT & O_JTV, WHV = OUT & O_HV;
  constexpr bool NEEDJ = WJ || WJV || WJTV, NEEDH = WH || WHV;
  constexpr HTmpl<M> HT{};
  constexpr int NHD = (M::NHD > 0) ? M::NHD : 1;
  extern __shared__ __align__(16) double sm[];   // staged rows: component k at euler_off(k) * TILE
  __shared__ double red[TILE];
  const bool sF = WF && a.f, sC = WC && a.c, sG = WG && a.g, sJ = WJ && a.jv, sH = WH && a.hv;
  const bool doH = sH || WHV;
  const int t = threadIdx.x;
  ModelConst K = launch_consts<M, PAR>(a);
  const int64_t N = a.N;
  const int64_t xN = (int64_t)NX * N;  // first entry of X_N
  for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * TILE;
    const int64_t j = r0 + t;
    const int nrows = (int)min((int64_t)TILE, max(N - r0, (int64_t)0));
    double objterm = 0.0;
    if (j < N) {
      double z[NZ], yb[NX], cqd[NZ], pa[NX], pb[NX], mjx[NX][M::MAXRX], mju[NX][M::MAXRU], hd[NHD];
      load_node<M>(a, j, z);
      if (NEEDH) {  // own rows' multipliers y_{k,j} (not the sum of two rows)
#pragma unroll
        for (int k = 0; k < NX; ++k) yb[k] = (doH && M::HK(k)) ? __ldg(a.y + a.nb + (int64_t)k * N + j) : 0.0;
        node_cq<M>(a, false, cqd);
      }
      M::template eval<WC, NEEDJ, NEEDH>(K, z, yb, cqd, pa, pb, mjx, mju, hd);
      if (sC) {
#pragma unroll
        for (int k = 0; k < NX; ++k) a.c[a.nb + (int64_t)k * N + j] = fsub(K, __ldg(a.x + NX * (j + 1) + k), pa[k]);
      }
      if (sJ) {
#pragma unroll
        for (int k = 0; k < NX; ++k) {
          double* rp = sm + euler_off<M>(k) * TILE + t * euler_count<M>(k);
#pragma unroll
          for (int e = 0; e < M::MAXRX; ++e)
            if (e < M::RX(k)) rp[e] = (M::XV(k, e) == k) ? (M::JZ(k, e) ? -1.0 : fma(mjx[k][e], K.one, -1.0)) : mjx[k][e];
          rp[M::RX(k)] = 1.0;
#pragma unroll
          for (int e = 0; e < M::MAXRU; ++e)
            if (e < M::RU(k)) rp[M::RX(k) + 1 + e] = mju[k][e];
        }
      }
      double vz[NZ];
      if (WJV || WHV) load_vz<M>(a, a.v, j, vz);
      if (WJV) {
        double A[NX], Bm[NX], mdp[NX];
        jv_node<M, false>(K, mjx, mju, mdp, 0.0, vz, A, Bm);
#pragma unroll
        for (int k = 0; k < NX; ++k)
          a.ojv[a.nb + (int64_t)k * N + j] = fadd(K, Bm[k], __ldg(a.v + NX * (j + 1) + k));
        if (j == 0) {
#pragma unroll
          for (int k = 0; k < NX; ++k) a.ojv[k] = vz[k];
        }
      }
      if (WJTV) {  // own rows only: wbar = w_{k,j}
        double wl[NX], wr[NX], o[NZ];
#pragma unroll
        for (int k = 0; k < NX; ++k) {
          const double* row = a.wv + a.nb + (int64_t)k * N;
          wl[k] = (j >= 1) ? __ldg(row + j - 1) : 0.0;
          wr[k] = __ldg(row + j);
        }
        jtv_node<M>(a, K, a.wv, j, tile == 0, mjx, mju, wl, wr, wr, o);  // CTA-uniform boundary flag
        store_nz<M>(a, a.ojtv, j, o);
      }
      if (WHV) {
        double o[NZ];
        hv_node<M>(a, K, hd, cqd, vz, o);
        store_nz<M>(a, a.ohv, j, o);
      }
      if (sH) {
#pragma unroll
        for (int e = 0; e < HT.n; ++e) {
          const int p = a.hpos[e];
          if (p >= 0) {
            const double val = (HT.dyn[e] >= 0) ? hd[HT.dyn[e] >= 0 ? HT.dyn[e] : 0] : cqd[HT.a[e]];
            if (HT.a[e] < NX) a.hv[j * a.hx + p] = val;
            else a.hv[a.hbase_u + j * a.hu + p] = val;
          }
        }
      }
      if (sG || sF) {
        if (a.has_ref) objterm = sG ? node_grad<M, true, true>(a, K, z, false, j) : node_grad<M, true, false>(a, K, z, false, j);
        else objterm = sG ? node_grad<M, false, true>(a, K, z, false, j) : node_grad<M, false, false>(a, K, z, false, j);
      }
      if (j == 0) {
#pragma unroll
        for (int k = 0; k < NX; ++k) {
          if (sC) a.c[k] = z[k];
          if (sJ) a.jv[k] = 1.0;
        }
      }
    } else if (r0 + TILE > N && j == N) {  // the last node: states only (CTA-uniform test first)
      if (sG) {
#pragma unroll
        for (int k = 0; k < NX; ++k) a.g[xN + k] = 0.0;
      }
      if (a.has_final) {
#pragma unroll
        for (int k = 0; k < NX; ++k) {
          if (sC) a.c[NX + k] = __ldg(a.x + xN + k);
          if (sJ) a.jv[NX + k] = 1.0;
          if (WJV) a.ojv[NX + k] = __ldg(a.v + xN + k);
        }
      }
      if (WJTV) {
#pragma unroll
        for (int k = 0; k < NX; ++k) {
          double o = __ldg(a.wv + a.nb + (int64_t)k * N + N - 1);
          if (a.has_final) o = fadd(K, o, __ldg(a.wv + NX + k));
          a.ojtv[xN + k] = o;
        }
      }
      if (WHV) {
#pragma unroll
        for (int k = 0; k < NX; ++k) a.ohv[xN + k] = 0.0;
      }
    }
    if (sJ) {  // copy-out of the staged rows: TMA bulk copies where aligned, else coalesced
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      bool bulk = false;
#pragma unroll
      for (int k = 0; k < NX; ++k) {
        const int cnt = euler_count<M>(k);
        const double* src = sm + euler_off<M>(k) * TILE;
        double* dst = a.jv + a.jbase[k] + r0 * cnt;
        const int total = nrows * cnt;
        const unsigned bytes = 8u * (unsigned)total;
        if (total > 0 && ((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src) | bytes) & 15u) == 0) {
          if (t == 0) {
            const unsigned saddr = static_cast<unsigned>(__cvta_generic_to_shared(src));
            asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                         :: "l"(dst), "r"(saddr), "r"(bytes) : "memory");
          }
          bulk = true;
        } else {
          for (int i = t; i < total; i += TILE) dst[i] = src[i];
        }
      }
      if (bulk && t == 0) {  // the rows must have been read before the next tile restages them
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
      }
    }
    if (sF) {
      const double ts = tile_sum<TILE>(objterm, red, K.one);
      if (t == 0) a.partials[tile] = ts;
    }
    __syncthreads();
  }
  if (sF) finish_tiles<TILE>(a.partials, a.ntiles, a.counter, a.f, 0.5, red);
}

template <class M, int TILE, unsigned OUT, bool PAR>
ocp_status launch_euler_k(ocp* h, NodeArgs<M>& a, cudaStream_t s) {
  a.ntiles = (h->N + 1 + TILE - 1) / TILE;
  if (a.ntiles > h->max_partials) return set_err(h, OCP_EDIM, "too many tiles for the reduction scratch");
  const size_t smem = (OUT & O_J) ? sizeof(double) * (size_t)euler_total<M>() * TILE : 0;
  auto kern = k_euler<M, TILE, OUT, PAR>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_err(h, e, "cudaFuncSetAttribute(euler)");
  }
  kern<<<(int)a.ntiles, TILE, smem, s>>>(a);
  return cuda_err(h, cudaGetLastError(), "k_euler launch");
}

template <class M, int TILE, unsigned OUT>
ocp_status launch_euler_t(ocp* h, NodeArgs<M>& a, cudaStream_t s) {
  // (under forward Euler the constraints alone run through the O_ALL kernel, null outputs skipped)
  if constexpr (M::HAS_DPARAM || (M::NP > 0 && OUT == O_ALL)) {
    if (a.p0_dev) return launch_euler_k<M, TILE, OUT, true>(h, a, s);
  } else {
    if (a.p0_dev) return set_err(h, OCP_EMODEL, "device parameters are not provided for this output set");
  }
  return launch_euler_k<M, TILE, OUT, false>(h, a, s);
}

template <class M>
void fill_euler_args(const ocp* h, double sigma, NodeArgs<M>& a) {
  fill_args<M>(h, sigma, a);
  M::host_consts(h->params.data(), h->h, a.K);   // the scheme's step is h (not h/2)
  a.B = 0;
  a.E = h->N + 1;
}

template <class M, int TILE>
ocp_status euler_eval_dispatch(ocp* h, unsigned out, const EvalCall& c, cudaStream_t s) {
  if (c.range) return set_err(h, OCP_EMODEL, "node ranges are provided for the trapezoidal scheme");
  NodeArgs<M> a;
  fill_euler_args<M>(h, c.sigma, a);
  a.x = c.x; a.y = c.y; a.f = c.f; a.c = c.c; a.g = c.g; a.jv = c.jv; a.hv = c.hv;
  a.v = c.vn; a.wv = c.vm; a.ojv = c.ojv; a.ojtv = c.ojtv; a.ohv = c.ohv;
  switch (out) {
    case O_STEP: return launch_euler_t<M, TILE, O_STEP>(h, a, s);
    case O_J | O_H: return launch_euler_t<M, TILE, O_J | O_H>(h, a, s);
    default: return launch_euler_t<M, TILE, O_ALL>(h, a, s);  // subsets: NULL outputs are skipped
  }
}

template <class M, int TILE>
ocp_status euler_prod_dispatch(ocp* h, const ProdCall& c, cudaStream_t s) {
  if (c.dmu || c.pdir != 0.0 || c.pdir_dev || c.mixw)
    return set_err(h, OCP_EMODEL, "parameter derivatives are provided for the trapezoidal scheme");
  if (!M::HAS_DPARAM && h->p0_dev)
    return set_err(h, OCP_EMODEL, "device parameters under forward Euler: the constraints only");
  NodeArgs<M> a;
  fill_euler_args<M>(h, c.sigma, a);
  a.x = c.x; a.y = c.y;
  if (c.kind == P_JPROD) { a.v = c.v; a.ojv = c.out; return launch_euler_t<M, TILE, O_JV>(h, a, s); }
  if (c.kind == P_JTPROD) { a.wv = c.v; a.ojtv = c.out; return launch_euler_t<M, TILE, O_JTV>(h, a, s); }
  a.v = c.v; a.ohv = c.out;
  return launch_euler_t<M, TILE, O_HV>(h, a, s);
}

template <class M, int TILE>
ocp_status node_eval_dispatch(ocp* h, unsigned out, const EvalCall& c, cudaStream_t s) {
  if (!M::HAS_DPARAM && h->p0_dev && out != O_C) return set_err(h, OCP_EMODEL, "device parameters: the constraints only");
  if (h->scheme == OCP_SCHEME_EULER) return euler_eval_dispatch<M, TILE>(h, out, c, s);
  switch (out) {
    case O_F: return launch_eval_t<M, TILE, 1, O_F>(h, c, s);
    case O_C: return launch_eval_t<M, TILE, 1, O_C>(h, c, s);
    case O_G: return launch_eval_t<M, TILE, 1, O_G>(h, c, s);
    case O_J: return launch_eval_t<M, TILE, 1, O_J>(h, c, s);
    case O_H: return launch_eval_t<M, TILE, 1, O_H>(h, c, s);
    case O_J | O_H: return launch_eval_t<M, TILE, 1, O_J | O_H>(h, c, s);
    case O_STEP: return launch_eval_t<M, TILE, 1, O_STEP>(h, c, s);
    default: return launch_eval_t<M, TILE, 1, O_ALL>(h, c, s);
  }
}

template <class M, int TILE, bool PAR>
cudaError_t node_prod_launch(ocp* h, const ProdCall& c, const NodeArgs<M>& a, cudaStream_t s) {
  auto go = [&](auto kern, int64_t units) {
    const int grid = occupancy_grid(h, (const void*)kern, TILE, 0, units);
    kern<<<grid, TILE, 0, s>>>(a);
  };
  // the parameter-direction and mixed terms of the double backward exist for the Van der Pol
  // model alone (the C-ABI rejects them for the others)
  constexpr bool VDP = M::HAS_DPARAM;
  if (c.kind == P_JPROD) {
    if (VDP && (c.pdir != 0.0 || c.pdir_dev)) go(k_node_jprod<M, TILE, VDP, PAR>, a.ntiles);
    else go(k_node_jprod<M, TILE, false, PAR>, a.ntiles);
  } else if (c.kind == P_JTPROD) {
    const int64_t blocks = (a.E - a.B + TILE - 1) / TILE;
    if (c.dmu) go(k_node_jtprod<M, TILE, true, PAR>, blocks);
    else go(k_node_jtprod<M, TILE, false, PAR>, blocks);
  } else {
    const int64_t blocks = (h->N + 1 + TILE - 1) / TILE;
    if (VDP && c.mixw && c.mixs) go(k_node_hprod<M, TILE, VDP, PAR>, blocks);
    else go(k_node_hprod<M, TILE, false, PAR>, blocks);
  }
  return cudaGetLastError();
}

template <class M, int TILE>
ocp_status node_prod_dispatch(ocp* h, const ProdCall& c, cudaStream_t s) {
  if (h->scheme == OCP_SCHEME_EULER) return euler_prod_dispatch<M, TILE>(h, c, s);
  NodeArgs<M> a;
  fill_args<M>(h, c.sigma, a);
  a.x = c.x; a.y = c.y; a.v = c.v; a.out = c.out; a.dmu = c.dmu;
  a.pdir = c.pdir; a.pdir_dev = c.pdir_dev; a.mixw = c.mixw; a.mixs = c.mixs;
  a.B = 0; a.E = h->N + 1;
  if (c.kind == P_JTPROD) { a.B = c.B; a.E = c.E < 0 ? h->N + 1 : c.E; }
  if (c.kind == P_JPROD) a.ntiles = (h->N + 1 + (TILE - 2)) / (TILE - 1);
  cudaError_t e;
  if (c.kind == P_JTPROD && c.dmu && (int64_t)npa<M>() * ((a.E - a.B + TILE - 1) / TILE) > h->max_partials)
    return set_err(h, OCP_EDIM, "too many tiles for the reduction scratch");
  if constexpr (M::NP > 0) {  // device-resident parameters (bound for one call or more)
    e = a.p0_dev ? node_prod_launch<M, TILE, true>(h, c, a, s) : node_prod_launch<M, TILE, false>(h, c, a, s);
  } else {
    e = node_prod_launch<M, TILE, false>(h, c, a, s);
  }
  return cuda_err(h, e, "node product launch");
}

}  // namespace ocpg
