// FP64 kernels for the heat-equation model (method of lines, n cells, one control):
//   f_k = (x_{k-1} - 2 x_k + x_{k+1}) / dx^2 - x_k^3,  ghost x_{-1} = u (Dirichlet control),
//   ghost x_n = x_{n-1} (homogeneous Neumann);  0-based cells k = 0..n-1.
// Per-cell derivatives (all other entries are the constant 1/dx^2 of the Laplacian):
//   df_k/dx_k = -2/dx^2 - 3 x_k^2   (k < n-1),   -1/dx^2 - 3 x_k^2   (k = n-1)
//   d2 f_k/dx_k^2 = -6 x_k.
// Row template of component k (the defect of cell k): X cells {k-1, k, k+1} within 0..n-1 on
// each side, plus the control for k = 0, so 6 entries per row except the last cell's 4.
//
// Work decomposition: a CTA covers 32 consecutive nodes (one per lane); in the evaluation and
// H v its 8 warps take the cells in groups of 8, while the J + H values, Jv and J^T w run two
// warps per CTA on units of 16 cells of a tile (four times as many CTAs, the same number on
// every SM).  Row-coupled outputs (defects, Jacobian rows) use tiles that overlap by one node
// (the CTA owns 31 of its 32 nodes); node-local products use disjoint tiles.
// The states of the tile's nodes are staged in shared memory with a padded row (n+1 doubles)
// so that lanes reading different nodes hit different banks; node-major outputs (Hessian
// diagonal, J^T w, H v) are staged the same way and stored with consecutive threads on
// consecutive addresses, except the gradient, stored by each lane for its eight cells.  Component-major outputs (defects, Jacobian rows, Jv)
// are consecutive across lanes and are stored directly or through a per-warp row buffer.
#include <cstring>
#include <type_traits>

#include "node_kernels.cuh"
#include "ocp_internal.h"

namespace ocpg {

constexpr int HEAT_MAXC = 128;
constexpr int HT_LANES = HEAT_TILE_NODES;
constexpr int HT_WARPS = 8;
constexpr int HT_THREADS = HT_LANES * HT_WARPS;

struct HeatArgs {
  const double* __restrict__ x;
  const double* __restrict__ y;
  const double* __restrict__ v;
  const double* __restrict__ v2;  // Jv and J^T w in one launch: the direction of J^T w
  double *f, *c, *g, *jv, *hv, *out;
  double* out2;                   // ... and J^T w
  double* out3;                   // Jv, J^T w and H v in one launch: H v (direction v, multipliers y)
  double* partials;
  unsigned* counter;
  int64_t N, nb, B, E, ntiles, uoff;
  int n, has_final, has_ref, hu;
  double hh, mhh, mhidx2;   // hh, -hh, -hh/dx^2
  double d_in, d_last;      // hh * 2/dx^2, hh * 1/dx^2  (diagonal constant of -hh df_k/dx_k)
  double di_m1, di_p1, dl_m1, dl_p1;  // d_in - 1, d_in + 1, d_last - 1, d_last + 1
  double h3, h6, hidx2;     // 3 hh, 6 hh, hh/dx^2
  double one, mz;           // 1.0 and -0.0 at run time: sums and products are issued as FMAs
  double cq_in[HEAT_MAXC + 1], cq_end[HEAT_MAXC + 1];
  double gq_in[HEAT_MAXC + 1], gq_end[HEAT_MAXC + 1];
  double ref[HEAT_MAXC + 1];
};

// Doubles of the first shared-memory region of k_heat_eval: the staged states (32 rows of n+1),
// and at least the 256 the objective's reductions use when they reuse it.
__host__ __device__ __forceinline__ int heat_xlen(int n) {
  return HT_LANES * (n + 1) > HT_THREADS ? HT_LANES * (n + 1) : HT_THREADS;
}

__device__ __forceinline__ int64_t heat_jbase(const HeatArgs& a, int k) { return a.nb + (int64_t)6 * k * a.N; }

// a + b, a - b, a * b as FMAs against run-time 1 and -0 (same rounding; faster on GB300's FP64 pipe)
__device__ __forceinline__ double hadd(const HeatArgs& a, double u, double v) { return fma(u, a.one, v); }
__device__ __forceinline__ double hsub(const HeatArgs& a, double u, double v) { return fma(-v, a.one, u); }
__device__ __forceinline__ double hmul(const HeatArgs& a, double u, double v) { return fma(u, v, a.mz); }

// Stage the states (and controls) of nodes [r0, r0+nn) into sX[t*(n+1) + k], sX[t*(n+1) + n] = u.
__device__ __forceinline__ void heat_stage(const HeatArgs& a, const double* __restrict__ src, int64_t r0, int nn,
                                           double* sX) {
  const int n = a.n, ld = n + 1;
  const int total = nn * n;
  const double* base = src + (int64_t)n * r0;
  for (int i = threadIdx.x; i < total; i += HT_THREADS) {
    const int t = i / n, k = i - t * n;
    sX[t * ld + k] = __ldg(base + i);
  }
  for (int t = threadIdx.x; t < nn; t += HT_THREADS) sX[t * ld + n] = __ldg(src + a.uoff + r0 + t);
}

// ======================================================================================
// Fused evaluation
// ======================================================================================

// Jacobian rows of cell k for the tile's nodes: the entries on x_k are -1 + dk (left node) and
// +1 + dk (right node), dk = 3 hh x_k^2 + d (d = hh 2/dx^2, or hh/dx^2 at the Neumann end),
// written fma(3 hh, x_k^2, d -+ 1); every other entry is the constant c = -hh/dx^2.  Lane t
// writes the whole row (k, r0 + t): its own left entry, the right entry of lane t+1 (shuffle),
// the constants; entries by position (left X cells, right X cells, then the control's left
// and right entries for k = 0):
//   k = 0:        [jl, c, jr', c, c, c]        interior:  [c, jl, c, c, jr', c]
//   k = n-1:      [c, jl, c, jr']
// A row is 48 (or 32) bytes: three (two) 16-byte stores when the component's rows start on a
// 16-byte boundary, scalar stores otherwise; consecutive lanes write consecutive rows.
__device__ __forceinline__ void heat_jrows(const HeatArgs& a, int k, bool LAST, int t, bool act, int nrows,
                                           int64_t r0, double x2) {
  const double jl = fma(a.h3, x2, LAST ? a.dl_m1 : a.di_m1);
  const double jr = fma(a.h3, x2, LAST ? a.dl_p1 : a.di_p1);
  const double jrn = __shfl_down_sync(0xffffffffu, jr, 1);   // the right node's entry on x_k
  if (!(act && t < nrows)) return;
  const double c = a.mhidx2;
  const int cnt = LAST ? 4 : 6;
  double* rp = a.jv + heat_jbase(a, k) + (r0 + t) * cnt;
  double v[6];
  if (k == 0) { v[0] = jl; v[1] = c; v[2] = jrn; v[3] = c; v[4] = c; v[5] = c; }
  else if (LAST) { v[0] = c; v[1] = jl; v[2] = c; v[3] = jrn; v[4] = c; v[5] = c; }
  else { v[0] = c; v[1] = jl; v[2] = c; v[3] = c; v[4] = jrn; v[5] = c; }
  if ((reinterpret_cast<uintptr_t>(rp) & 15u) == 0) {
    double2* r2 = reinterpret_cast<double2*>(rp);
    r2[0] = make_double2(v[0], v[1]);
    r2[1] = make_double2(v[2], v[3]);
    if (!LAST) r2[2] = make_double2(v[4], v[5]);
  } else {
#pragma unroll
    for (int e = 0; e < 6; ++e)
      if (e < cnt) rp[e] = v[e];
  }
}

// boundary rows X_{0,k} (and X_{N,k}): one constant entry each
__device__ __forceinline__ void heat_jbound(const HeatArgs& a, int k, int64_t j) {
  if (j == 0) a.jv[k] = 1.0;
  if (a.has_final && j == a.N) a.jv[a.n + k] = 1.0;
}

// Hessian diagonal of cell k at node j: 6 hh ybar_k x_k + the objective's sigma w q_k
// (yl, yr = y_{k,j-1}, y_{k,j}, zero beyond the first and last rows)
__device__ __forceinline__ double heat_hdiag_y(const HeatArgs& a, int k, bool endp, double xk, double yl, double yr) {
  const double ty = hmul(a, a.h6, hadd(a, yl, yr));
  return fma(ty, xk, endp ? a.cq_end[k] : a.cq_in[k]);
}
__device__ __forceinline__ double heat_hdiag(const HeatArgs& a, int k, int64_t j, bool endp, double xk) {
  const double yl = (j >= 1) ? __ldg(a.y + a.nb + (int64_t)k * a.N + j - 1) : 0.0;
  const double yr = (j < a.N) ? __ldg(a.y + a.nb + (int64_t)k * a.N + j) : 0.0;
  return heat_hdiag_y(a, k, endp, xk, yl, yr);
}

// gradient entry of cell k at node j and its objective term
__device__ __forceinline__ void heat_grad(const HeatArgs& a, int k, int64_t j, bool endp, double xk, bool WG, bool WF,
                                          double& objacc) {
  const double d = a.has_ref ? hsub(a, xk, a.ref[k]) : xk;
  const double gk = hmul(a, endp ? a.gq_end[k] : a.gq_in[k], d);
  if (WF) objacc = fma(gk, d, objacc);
  if (WG) a.g[(int64_t)a.n * j + k] = gk;
}

template <unsigned OUT>
__global__ void __launch_bounds__(HT_THREADS, (OUT & O_C) ? 5 : 8) k_heat_eval(const __grid_constant__ HeatArgs a) {
  constexpr bool CF = OUT & O_F, CC = OUT & O_C, CG = OUT & O_G, CJ = OUT & O_J, CH = OUT & O_H;
  // the full kernel also serves output subsets: NULL outputs are skipped
  const bool WF = CF && a.f, WC = CC && a.c, WG = CG && a.g, WJ = CJ && a.jv, WH = CH && a.hv;
  extern __shared__ __align__(16) double sm[];
  const int n = a.n, ld = n + 1;
  // shared memory: states, then only the staging buffers this variant needs.  The gradient
  // is stored straight from the cell loop (a lane's eight cells of a group fill whole 32-byte
  // sectors) and the objective's reduction reuses the states' buffer once the tile's stores
  // are done: the full evaluation fits five CTAs per SM (one wave of 646 tiles at N = 2e4).
  double* sX = sm;                                             // 32 * ld
  double* sN = sX + heat_xlen(n);                              // Hessian diagonal, 31 * ld
  double* red = sX;                                            // reduction, 256 (after the stores)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double objacc = 0.0;

  for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const int64_t r0 = a.B + tile * (HT_LANES - 1);
    const int64_t own_end = min(r0 + HT_LANES - 1, a.E);
    const int64_t row_end = min(own_end, a.N);
    const int64_t eval_end = row_end + 1;
    const int nn = (int)(eval_end - r0);
    const int nown = (int)(own_end - r0);
    const int nrows = (int)max(row_end - r0, (int64_t)0);
    const int t = lane;
    const int64_t j = r0 + t;
    const bool act = t < nn;
    const bool own = t < nown;
    const bool endp = (j == 0) || (j == a.N);
    heat_stage(a, a.x, r0, nn, sX);
    __syncthreads();
    // ---- Hessian diagonal of every owned (node, cell), elementwise: warps take whole cells
    // (lanes = nodes, the multipliers' rows coalesced), so no load waits inside the cell loop
    // (measured: the separate pass speeds up the full evaluation; J + H alone is faster with
    // the diagonal computed in its cell loop)
    if (CC && WH && own) {
#pragma unroll 2
      for (int k = warp; k < n; k += HT_WARPS) sN[t * ld + k] = heat_hdiag(a, k, j, endp, sX[t * ld + k]);
    }

    // ---- control entries (warp 0): gradient, objective, Hessian (u,u)
    if (warp == 0 && own) {
      const double u = sX[t * ld + n];
      if (WG || WF) {
        const double d = a.has_ref ? hsub(a, u, a.ref[n]) : u;
        const double gu = hmul(a, endp ? a.gq_end[n] : a.gq_in[n], d);
        if (WG) a.g[a.uoff + j] = gu;
        if (WF) objacc = fma(gu, d, objacc);
      }
      if (WH && a.hu) a.hv[(int64_t)n * (a.N + 1) + j] = endp ? a.cq_end[n] : a.cq_in[n];
    }

    const int ngroups = (n + 7) / 8;
    if constexpr (CC) {
      // One cell k of the tile's nodes; LAST: k is the Neumann end n-1.  The end cell is
      // peeled out of the loop so that its Laplacian and diagonal constant are compile-time
      // choices: a run-time select between two FP64 results issues both on every cell.
      auto cell = [&](const int k, auto last_tag) {
        constexpr bool LAST = decltype(last_tag)::value;
        double xk = 0.0, xl = 0.0, xr = 0.0;
        if (act) {
          xk = sX[t * ld + k];
          xl = (k == 0) ? sX[t * ld + n] : sX[t * ld + k - 1];
          xr = LAST ? xk : sX[t * ld + k + 1];
        }
        const double x2 = hmul(a, xk, xk);
        if (WJ) heat_jrows(a, k, LAST, t, act, nrows, r0, x2);
        if (WJ && own) heat_jbound(a, k, j);
        if (WC) {
          // hh f_k = hh (lap / dx^2 - x^3)
          // pa = x + hh f, pb = x - hh f, with hh f = hh/dx^2 lap - hh x^3
          const double lap = LAST ? hsub(a, xl, xk) : fma(-2.0, xk, hadd(a, xl, xr));
          const double x3 = hmul(a, x2, xk);
          const double pa = fma(a.hidx2, lap, fma(a.mhh, x3, xk));
          const double pb = fma(-a.hidx2, lap, fma(a.hh, x3, xk));
          const double nb = __shfl_down_sync(0xffffffffu, pb, 1);
          if (t < nrows) a.c[a.nb + (int64_t)k * a.N + j] = hsub(a, nb, pa);
          if (own && j == 0) a.c[k] = xk;
          if (own && a.has_final && j == a.N) a.c[n + k] = xk;
        }
        if (own && (WG || WF)) heat_grad(a, k, j, endp, xk, WG, WF, objacc);
      };
      for (int gi = warp; gi < ngroups; gi += HT_WARPS) {
        const int k0 = gi * 8, k1 = min(k0 + 8, n);
        const int kin = min(k1, n - 1);  // interior cells of the group: k0 .. kin-1
#pragma unroll 1
        for (int k = k0; k < kin; ++k) cell(k, std::false_type{});
        if (k1 == n) cell(n - 1, std::true_type{});
      }
    } else {
      // without the constraints one loop body for every cell (smaller and measured faster)
      for (int gi = warp; gi < ngroups; gi += HT_WARPS) {
        const int k0 = gi * 8, k1 = min(k0 + 8, n);
        for (int k = k0; k < k1; ++k) {
          const bool last = (k == n - 1);
          double xk = 0.0;
          if (act) xk = sX[t * ld + k];
          if (WJ) heat_jrows(a, k, last, t, act, nrows, r0, hmul(a, xk, xk));
          if (WJ && own) heat_jbound(a, k, j);
          if (own && WH) sN[t * ld + k] = heat_hdiag(a, k, j, endp, xk);
          if (own && (WG || WF)) heat_grad(a, k, j, endp, xk, WG, WF, objacc);
        }
      }
    }
    __syncthreads();
    if (WH) {
      const int total = nown * n;
      double* dst = a.hv + (int64_t)n * r0;
      for (int i = threadIdx.x; i < total; i += HT_THREADS) {
        const int tt = i / n, k = i - tt * n;
        dst[i] = sN[tt * ld + k];
      }
    }
    if (WF) {
      __syncthreads();  // red is the states' buffer, read by the loop above
      const double ts = tile_sum<HT_THREADS>(objacc, red, a.one);
      if (threadIdx.x == 0) a.partials[tile] = ts;
      objacc = 0.0;
    }
    __syncthreads();
  }
  if (WF) finish_tiles<HT_THREADS>(a.partials, a.ntiles, a.counter, a.f, 0.5, red);
}

// ======================================================================================
// Jacobian and Hessian values alone (no objective, defects or gradient).  Each entry depends on
// its own cell only, so a CTA of two warps takes one tile's 32 nodes (31 owned) and 16 of its
// cells, eight per warp: a problem splits into ceil(n/16) times as many CTAs as tiles, spread
// evenly over the SMs (at N = 2e4 and 64 cells: 2584 CTAs, 17 per SM in one wave, where the
// 646 CTAs of whole tiles put 4 on some SMs and 5 on others).  Every entry is computed by the
// same expressions as in k_heat_eval, so the values are bit-identical.
// ======================================================================================
constexpr int HJ_CELLS = 16, HJ_WARPS = 2, HJ_THREADS = 32 * HJ_WARPS, HJ_LD = HJ_CELLS + 1;

template <unsigned OUT>
__global__ void __launch_bounds__(HJ_THREADS, 18) k_heat_jh(const __grid_constant__ HeatArgs a, int cgroups) {
  constexpr bool CJ = OUT & O_J, CH = OUT & O_H;
  const bool WJ = CJ && a.jv, WH = CH && a.hv;
  // the states of the unit's cells, node-major in padded rows, overwritten in place by the
  // Hessian diagonal; the multipliers y_{k, r0-1 .. r0+30} of its cells, cell-major
  __shared__ double sX[HT_LANES * HJ_LD];
  __shared__ double sY[HJ_CELLS * HT_LANES];
  const int n = a.n;
  const int t = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t units = a.ntiles * cgroups;
  for (int64_t unit = blockIdx.x; unit < units; unit += gridDim.x) {
    const int64_t tile = unit / cgroups;
    const int c0 = (int)(unit - tile * cgroups) * HJ_CELLS;
    const int nc = min(HJ_CELLS, n - c0);
    const int64_t r0 = a.B + tile * (HT_LANES - 1);
    const int64_t own_end = min(r0 + HT_LANES - 1, a.E);
    const int64_t row_end = min(own_end, a.N);
    const int nn = (int)(row_end + 1 - r0);
    const int nown = (int)(own_end - r0);
    const int nrows = (int)max(row_end - r0, (int64_t)0);
    const int64_t j = r0 + t;
    const bool act = t < nn;
    const bool own = t < nown;
    const bool endp = (j == 0) || (j == a.N);
    for (int i = threadIdx.x; i < nn * nc; i += HJ_THREADS) {
      const int tt = i / nc, kk = i - tt * nc;
      sX[tt * HJ_LD + kk] = __ldg(a.x + (int64_t)n * (r0 + tt) + c0 + kk);
    }
    if (WH) {
      // rows outside [0, N) stage as zero: y_{k,j-1} for j = 0 and y_{k,j} for j = N
      for (int i = threadIdx.x; i < nc * HT_LANES; i += HJ_THREADS) {
        const int kk = i / HT_LANES;
        const int64_t jj = r0 - 1 + (i - kk * HT_LANES);
        sY[i] = (jj >= 0 && jj < a.N) ? __ldg(a.y + a.nb + (int64_t)(c0 + kk) * a.N + jj) : 0.0;
      }
    }
    __syncthreads();
    // the control's Hessian entry (u, u), by the unit of the first cells
    if (c0 == 0 && warp == 0 && own && WH && a.hu) a.hv[(int64_t)n * (a.N + 1) + j] = endp ? a.cq_end[n] : a.cq_in[n];
    const int k1 = min(8 * warp + 8, nc);
    for (int kk = 8 * warp; kk < k1; ++kk) {
      const int k = c0 + kk;
      double xk = 0.0;
      if (act) xk = sX[t * HJ_LD + kk];
      if (WJ) heat_jrows(a, k, k == n - 1, t, act, nrows, r0, hmul(a, xk, xk));
      if (WJ && own) heat_jbound(a, k, j);
      // an owned lane t <= 30 reads the multipliers of rows j-1 and j at positions t and t+1
      if (own && WH) sX[t * HJ_LD + kk] = heat_hdiag_y(a, k, endp, xk, sY[kk * HT_LANES + t], sY[kk * HT_LANES + t + 1]);
    }
    __syncthreads();
    if (WH) {
      double* dst = a.hv + (int64_t)n * r0 + c0;
      for (int i = threadIdx.x; i < nown * nc; i += HJ_THREADS) {
        const int tt = i / nc, kk = i - tt * nc;
        dst[(int64_t)n * tt + kk] = sX[tt * HJ_LD + kk];
      }
    }
    __syncthreads();
  }
}

// ======================================================================================
// H v (node-local):    out_a = (2 sigma w q_a + 6 hh ybar_a x_a) v_a,  out_u = 2 sigma w r v_u
// (whole tiles of 32 nodes and their 64 cells: measured faster than the 16-cell units of the
// other products, 23.3 against 24.3 us at N = 2e4, 39.4 against 41.1 at N = 5e4); at most 51
// registers: five CTAs per SM, one wave of 626 tiles at N = 2e4 (measured faster)
// ======================================================================================
__global__ void __launch_bounds__(HT_THREADS, 5) k_heat_hprod(const __grid_constant__ HeatArgs a) {
  extern __shared__ __align__(16) double sm[];
  const int n = a.n, ld = n + 1;
  double* sX = sm;
  double* sV = sX + HT_LANES * ld;  // the direction
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * HT_LANES;
    const int nn = (int)min((int64_t)HT_LANES, a.N + 1 - r0);
    const int t = lane;
    const int64_t j = r0 + t;
    const bool act = t < nn;
    const bool endp = (j == 0) || (j == a.N);
    heat_stage(a, a.x, r0, nn, sX);
    heat_stage(a, a.v, r0, nn, sV);
    __syncthreads();
    const int ngroups = (n + 7) / 8;
    for (int gi = warp; gi < ngroups; gi += HT_WARPS) {
      const int k0 = gi * 8, k1 = min(k0 + 8, n);
      // elementwise: the group's multiplier rows are loaded before any arithmetic needs them
      double yl[8], yr[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int k = k0 + q;
        yl[q] = (act && k < k1 && j >= 1) ? __ldg(a.y + a.nb + (int64_t)k * a.N + j - 1) : 0.0;
        yr[q] = (act && k < k1 && j < a.N) ? __ldg(a.y + a.nb + (int64_t)k * a.N + j) : 0.0;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int k = k0 + q;
        if (act && k < k1) {
          const double xk = sX[t * ld + k];
          const double hk = fma(hmul(a, a.h6, hadd(a, yl[q], yr[q])), xk, endp ? a.cq_end[k] : a.cq_in[k]);
          sX[t * ld + k] = hmul(a, hk, sV[t * ld + k]);  // in place: x no longer needed for cell k
        }
      }
    }
    if (warp == 0 && act) {
      const double cu = a.hu ? (endp ? a.cq_end[n] : a.cq_in[n]) : 0.0;
      sX[t * ld + n] = hmul(a, cu, sV[t * ld + n]);
    }
    __syncthreads();
    {
      const int total = nn * n;
      double* dst = a.out + (int64_t)n * r0;
      for (int i = threadIdx.x; i < total; i += HT_THREADS) {
        const int tt = i / n, k = i - tt * n;
        dst[i] = sX[tt * ld + k];
      }
      for (int tt = threadIdx.x; tt < nn; tt += HT_THREADS) a.out[a.uoff + r0 + tt] = sX[tt * ld + n];
    }
    __syncthreads();
  }
}

// ======================================================================================
// Jv and J^T w on units of one tile and 16 cells (two warps of 8 cells each, as in k_heat_jh),
// so that the work spreads evenly over the SMs (at N = 2e4: Jv 35.0 -> 31.4 us, J^T w 31.8 ->
// 28.9 us, against whole tiles of 32 nodes and 64 cells).
//   Jv:     p_k(j) = -hh grad f_k(z_j) . v_{z_j};
//           row (k,j) = (p_k(j) - v_{X_j,k}) + (p_k(j+1) + v_{X_{j+1},k})
//           on tiles overlapping by one node (its rows couple nodes j and j+1); the direction of
//           cells c0-1 .. c0+16 is staged, the control's in place of cell -1.
//   J^T w:  out_a = (w_{a,j-1} - w_{a,j}) + wbar_a dd_a - hh/dx^2 (wbar_{a-1} + wbar_{a+1}),
//           out_u = -hh/dx^2 wbar_0  (dd_a = -hh df_a/dx_a), node-local on disjoint tiles; the
//           result is staged and stored node by node in runs of the unit's cells.
//   Both (the heat model's fused step): the two products of the same unit in one launch, on the
//           tiles of Jv; J^T w for the owned nodes, its result written over the staged states
//           once Jv has read them.  All three: H v of the owned nodes as well, each entry formed
//           in Jv's cell loop from the same state and direction values and stored by its lane.
//           Each entry by the same expressions as the separate launches.
// ======================================================================================
enum : int { HP_JPROD = 0, HP_JTPROD = 1, HP_BOTH = 2, HP_ALL3 = 3 };
constexpr int HP_LDV = HJ_CELLS + 3;  // padded row of the staged direction (or J^T w result)

template <int KIND>
__global__ void __launch_bounds__(HJ_THREADS, 18) k_heat_prod_unit(const __grid_constant__ HeatArgs a, int cgroups) {
  constexpr bool ALL3 = KIND == HP_ALL3, BOTH = KIND == HP_BOTH || ALL3;
  constexpr bool JP = KIND == HP_JPROD || BOTH, JT = KIND == HP_JTPROD || BOTH;
  constexpr int LDV = JP ? HP_LDV : HJ_LD;
  __shared__ double sX[HT_LANES * HJ_LD];  // states of the unit's cells (both: then the J^T w result)
  __shared__ double sV[HT_LANES * LDV];    // Jv: the direction; J^T w alone: the result
  double* const sO = BOTH ? sX : sV;       // the J^T w result (row length HJ_LD either way)
  const double* const wv = BOTH ? a.v2 : a.v;
  double* const wout = BOTH ? a.out2 : a.out;
  const int n = a.n;
  const int t = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t units = a.ntiles * cgroups;
  for (int64_t unit = blockIdx.x; unit < units; unit += gridDim.x) {
    const int64_t tile = unit / cgroups;
    const int c0 = (int)(unit - tile * cgroups) * HJ_CELLS;
    const int nc = min(HJ_CELLS, n - c0);
    const int kb = 8 * warp, ke = min(8 * warp + 8, nc);  // this warp's cells c0 + [kb, ke)
    int64_t r0;
    int nn, nrows = 0, nown = 0;
    bool bnd = false;
    if (JP) {
      r0 = tile * (HT_LANES - 1);
      const int64_t own_end = min(r0 + HT_LANES - 1, a.N + 1);
      const int64_t row_end = min(own_end, a.N);
      nn = (int)(row_end + 1 - r0);
      nrows = (int)max(row_end - r0, (int64_t)0);
      nown = (int)(own_end - r0);
    } else {
      r0 = tile * HT_LANES;
      nn = (int)min((int64_t)HT_LANES, a.N + 1 - r0);
      bnd = (tile == 0) || (r0 + HT_LANES > a.N);
    }
    if (BOTH) bnd = (r0 == 0) || (r0 + nown == a.N + 1);  // the tile holds node 0 or node N
    const int64_t j = r0 + t;
    const bool act = t < nn;
    const bool jown = BOTH ? (t < nown) : act;  // J^T w: the owned nodes
    for (int i = threadIdx.x; i < nn * nc; i += HJ_THREADS) {
      const int tt = i / nc, kk = i - tt * nc;
      sX[tt * HJ_LD + kk] = __ldg(a.x + (int64_t)n * (r0 + tt) + c0 + kk);
    }
    if (JP) {
      const int w = nc + 2;  // cells c0-1 .. c0+nc at positions 0 .. nc+1
      for (int i = threadIdx.x; i < nn * w; i += HJ_THREADS) {
        const int tt = i / w, e = i - tt * w, k = c0 - 1 + e;
        double val = 0.0;
        if (k < 0) val = __ldg(a.v + a.uoff + r0 + tt);
        else if (k < n) val = __ldg(a.v + (int64_t)n * (r0 + tt) + k);
        sV[tt * HP_LDV + e] = val;
      }
    }
    __syncthreads();
    if (JP) {
      const bool endp = (j == 0) || (j == a.N);
      if (ALL3 && c0 == 0 && warp == 0 && jown) {  // H v, the control: 2 sigma w r v_u
        const double cu = a.hu ? (endp ? a.cq_end[n] : a.cq_in[n]) : 0.0;
        a.out3[a.uoff + j] = hmul(a, cu, sV[t * HP_LDV]);
      }
      for (int kk = kb; kk < ke; ++kk) {
        const int k = c0 + kk;
        double p = 0.0, vk = 0.0;
        if (act) {
          const double xk = sX[t * HJ_LD + kk];
          const bool last = (k == n - 1);
          if (ALL3 && jown) {  // H v: (2 sigma w q_k + 6 hh ybar_k x_k) v_k
            const double* yrow = a.y + a.nb + (int64_t)k * a.N;
            const double yl = (j >= 1) ? __ldg(yrow + j - 1) : 0.0;
            const double yr = (j < a.N) ? __ldg(yrow + j) : 0.0;
            const double hk = fma(hmul(a, a.h6, hadd(a, yl, yr)), xk, endp ? a.cq_end[k] : a.cq_in[k]);
            a.out3[(int64_t)n * j + k] = hmul(a, hk, sV[t * HP_LDV + kk + 1]);
          }
          vk = sV[t * HP_LDV + kk + 1];
          const double vl = sV[t * HP_LDV + kk];  // cell k-1, or the control for k = 0
          const double dk = fma(a.h3, hmul(a, xk, xk), last ? a.d_last : a.d_in);
          const double nsum = last ? vl : hadd(a, vl, sV[t * HP_LDV + kk + 2]);
          p = fma(a.mhidx2, nsum, hmul(a, dk, vk));
        }
        const double right = __shfl_down_sync(0xffffffffu, hadd(a, p, vk), 1);
        if (t < nrows) a.out[a.nb + (int64_t)k * a.N + j] = hadd(a, hsub(a, p, vk), right);
        if (act && j == 0) a.out[k] = vk;
        if (act && a.has_final && j == a.N && t < nown) a.out[n + k] = vk;
      }
    }
    if (JT && kb < ke) {
      // wbar of cells k0-1 .. k1 (clamped), rolling window
      auto wbar = [&](int k, double& wl, double& wr) {
        const double* row = wv + a.nb + (int64_t)k * a.N;
        wl = (j >= 1) ? __ldg(row + j - 1) : 0.0;
        wr = (j < a.N) ? __ldg(row + j) : 0.0;
      };
      const int k0 = c0 + kb, k1 = c0 + ke;
      double wbm = 0.0, wbc = 0.0, wbp = 0.0, wlc = 0.0, wrc = 0.0;
      if (jown) {
        if (k0 > 0) { double l2, r2; wbar(k0 - 1, l2, r2); wbm = hadd(a, l2, r2); }
        wbar(k0, wlc, wrc);
        wbc = hadd(a, wlc, wrc);
        if (k0 == 0) wout[a.uoff + j] = hmul(a, a.mhidx2, wbc);  // control column: -hh/dx^2 wbar_0
      }
      for (int k = k0; k < k1; ++k) {
        if (jown) {
          double wlp = 0.0, wrp = 0.0;
          if (k + 1 < n) { wbar(k + 1, wlp, wrp); wbp = hadd(a, wlp, wrp); } else wbp = 0.0;
          const double xk = sX[t * HJ_LD + (k - c0)];
          const bool last = (k == n - 1);
          const double dk = fma(a.h3, hmul(a, xk, xk), last ? a.d_last : a.d_in);
          double s = fma(wbc, dk, hsub(a, wlc, wrc));
          s = fma(a.mhidx2, hadd(a, wbm, wbp), s);
          if (bnd) {  // only the CTAs holding node 0 or node N (uniform branch)
            if (j == 0) s = hadd(a, s, __ldg(wv + k));
            if (a.has_final && j == a.N) s = hadd(a, s, __ldg(wv + n + k));
          }
          sO[t * HJ_LD + (k - c0)] = s;
          wbm = wbc; wbc = wbp; wlc = wlp; wrc = wrp;
        }
      }
    }
    __syncthreads();
    if (JT) {
      // node-major results of the unit's cells, in runs of nc per node
      double* dst = wout + (int64_t)n * r0 + c0;
      const int nst = BOTH ? nown : nn;
      for (int i = threadIdx.x; i < nst * nc; i += HJ_THREADS) {
        const int tt = i / nc, kk = i - tt * nc;
        dst[(int64_t)n * tt + kk] = sO[tt * HJ_LD + kk];
      }
    }
    __syncthreads();
  }
}

// ======================================================================================
// Host side
// ======================================================================================
static void heat_fill(const ocp* h, double sigma, HeatArgs& a) {
  memset(&a, 0, sizeof(a));
  const int n = h->nx;
  const double idx2 = (double)n * (double)n;  // 1/dx^2 with dx = 1/n
  a.N = h->N;
  a.nb = h->pat.nb;
  a.uoff = (int64_t)n * (h->N + 1);
  a.n = n;
  a.has_final = h->has_final;
  a.has_ref = h->has_ref;
  a.hu = h->pat.hu;
  a.hh = h->hh;
  a.mhh = -h->hh;
  a.mhidx2 = -h->hh * idx2;
  a.hidx2 = h->hh * idx2;
  a.d_in = h->hh * (2.0 * idx2);
  a.d_last = h->hh * idx2;
  a.di_m1 = a.d_in - 1.0;
  a.di_p1 = a.d_in + 1.0;
  a.dl_m1 = a.d_last - 1.0;
  a.dl_p1 = a.d_last + 1.0;
  a.h3 = 3.0 * h->hh;
  a.h6 = 6.0 * h->hh;
  a.one = 1.0;
  a.mz = -0.0;
  for (int v = 0; v <= n; ++v) {
    const double w = v < n ? h->q[v] : h->r[0];
    a.gq_in[v] = 2.0 * h->h * w;
    a.gq_end[v] = h->h * w;
    a.cq_in[v] = sigma * (2.0 * h->h * w);
    a.cq_end[v] = sigma * (h->h * w);
    a.ref[v] = v < n ? h->xref[v] : h->uref[0];
  }
  a.partials = h->d_partials;
  a.counter = h->d_counter;
}

template <unsigned OUT>
static ocp_status heat_eval_t(ocp* h, const EvalCall& c, cudaStream_t s) {
  HeatArgs a;
  heat_fill(h, c.sigma, a);
  a.x = c.x; a.y = c.y; a.f = c.f; a.c = c.c; a.g = c.g; a.jv = c.jv; a.hv = c.hv;
  a.B = c.B; a.E = c.E;
  const int64_t nodes = c.E - c.B;
  a.ntiles = (nodes + (HT_LANES - 2)) / (HT_LANES - 1);
  if (a.ntiles < 1) a.ntiles = 1;
  if (a.ntiles > h->max_partials) return set_err(h, OCP_EDIM, "too many tiles for the reduction scratch");
  const int ld = h->nx + 1;
  const size_t smem = sizeof(double) * ((size_t)heat_xlen(h->nx) + ((OUT & O_H) ? (HT_LANES - 1) * ld : 0));
  auto kern = k_heat_eval<OUT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_err(h, e, "cudaFuncSetAttribute(heat)");
  const int grid = occupancy_grid(h, (const void*)kern, HT_THREADS, smem, a.ntiles);
  if (grid <= 0) return set_err(h, OCP_ECUDA, "occupancy query failed");
  kern<<<grid, HT_THREADS, smem, s>>>(a);
  return cuda_err(h, cudaGetLastError(), "k_heat_eval launch");
}

// Jacobian and / or Hessian values alone: units of one tile and 16 cells (k_heat_jh)
template <unsigned OUT>
static ocp_status heat_jh_t(ocp* h, const EvalCall& c, cudaStream_t s) {
  HeatArgs a;
  heat_fill(h, c.sigma, a);
  a.x = c.x; a.y = c.y; a.jv = c.jv; a.hv = c.hv;
  a.B = c.B; a.E = c.E;
  const int64_t nodes = c.E - c.B;
  a.ntiles = (nodes + (HT_LANES - 2)) / (HT_LANES - 1);
  if (a.ntiles < 1) a.ntiles = 1;
  const int cgroups = (h->nx + HJ_CELLS - 1) / HJ_CELLS;
  auto kern = k_heat_jh<OUT>;
  const int grid = occupancy_grid(h, (const void*)kern, HJ_THREADS, 0, a.ntiles * cgroups);
  if (grid <= 0) return set_err(h, OCP_ECUDA, "occupancy query failed");
  kern<<<grid, HJ_THREADS, 0, s>>>(a, cgroups);
  return cuda_err(h, cudaGetLastError(), "k_heat_jh launch");
}

ocp_status heat_eval(ocp* h, unsigned out, const EvalCall& c, cudaStream_t s) {
  switch (out) {
    case O_F: return heat_eval_t<O_F>(h, c, s);
    case O_C: return heat_eval_t<O_C>(h, c, s);
    case O_G: return heat_eval_t<O_G>(h, c, s);
    case O_J: return heat_jh_t<O_J>(h, c, s);
    case O_H: return heat_jh_t<O_H>(h, c, s);
    case O_J | O_H: return heat_jh_t<O_J | O_H>(h, c, s);
    default: return heat_eval_t<O_ALL>(h, c, s);
  }
}

// Jv (jp.v -> jp.out), J^T w (jt.v -> jt.out) and, with hp, H v (hp.y, hp.sigma, the direction
// jp.v -> hp.out) of the heat model in one launch (the fused step)
ocp_status heat_prod2(ocp* h, const ProdCall& jp, const ProdCall& jt, const ProdCall* hp, cudaStream_t s) {
  HeatArgs a;
  heat_fill(h, hp ? hp->sigma : 1.0, a);
  a.x = jp.x; a.v = jp.v; a.out = jp.out; a.v2 = jt.v; a.out2 = jt.out;
  if (hp) { a.y = hp->y; a.out3 = hp->out; }
  const int cgroups = (h->nx + HJ_CELLS - 1) / HJ_CELLS;
  a.ntiles = (h->N + 1 + (HT_LANES - 2)) / (HT_LANES - 1);
  const void* k = hp ? (const void*)k_heat_prod_unit<HP_ALL3> : (const void*)k_heat_prod_unit<HP_BOTH>;
  const int grid = occupancy_grid(h, k, HJ_THREADS, 0, a.ntiles * cgroups);
  if (grid <= 0) return set_err(h, OCP_ECUDA, "occupancy query failed");
  if (hp) k_heat_prod_unit<HP_ALL3><<<grid, HJ_THREADS, 0, s>>>(a, cgroups);
  else k_heat_prod_unit<HP_BOTH><<<grid, HJ_THREADS, 0, s>>>(a, cgroups);
  return cuda_err(h, cudaGetLastError(), "heat product launch");
}

ocp_status heat_prod(ocp* h, const ProdCall& c, cudaStream_t s) {
  HeatArgs a;
  heat_fill(h, c.sigma, a);
  a.x = c.x; a.y = c.y; a.v = c.v; a.out = c.out;
  if (c.kind == P_HPROD) {
    a.ntiles = (h->N + 1 + HT_LANES - 1) / HT_LANES;
    const size_t smem = sizeof(double) * (size_t)HT_LANES * (h->nx + 1) * 2;  // states and direction
    auto k = k_heat_hprod;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_err(h, e, "cudaFuncSetAttribute(heat hprod)");
    const int grid = occupancy_grid(h, (const void*)k, HT_THREADS, smem, a.ntiles);
    k<<<grid, HT_THREADS, smem, s>>>(a);
    return cuda_err(h, cudaGetLastError(), "heat product launch");
  }
  const int cgroups = (h->nx + HJ_CELLS - 1) / HJ_CELLS;
  if (c.kind == P_JPROD) a.ntiles = (h->N + 1 + (HT_LANES - 2)) / (HT_LANES - 1);
  else a.ntiles = (h->N + 1 + HT_LANES - 1) / HT_LANES;
  const void* k = (c.kind == P_JPROD) ? (const void*)k_heat_prod_unit<HP_JPROD> : (const void*)k_heat_prod_unit<HP_JTPROD>;
  const int grid = occupancy_grid(h, k, HJ_THREADS, 0, a.ntiles * cgroups);
  if (grid <= 0) return set_err(h, OCP_ECUDA, "occupancy query failed");
  if (c.kind == P_JPROD) k_heat_prod_unit<HP_JPROD><<<grid, HJ_THREADS, 0, s>>>(a, cgroups);
  else k_heat_prod_unit<HP_JTPROD><<<grid, HJ_THREADS, 0, s>>>(a, cgroups);
  return cuda_err(h, cudaGetLastError(), "heat product launch");
}

}  // namespace ocpg
