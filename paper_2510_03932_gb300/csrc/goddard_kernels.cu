// Fused FP64 kernels of the Goddard rocket problem (paper appendix) with a free final time.
//
// The transcription is the trapezoidal one of the other models (paper Sec. 5), with the
// horizon tf read from x[n-1] when it is free (h = tf / N).  tf couples every node:
//   - each defect row (k, j) ends with its tf entry  -(f_k(z_j) + f_k(z_{j+1})) / (2N);
//   - the Lagrangian Hessian ends with the tf row  -(1/(2N)) sum_k ybar_{j,k} grad f_k(z_j)
//     (c is linear in tf and there is no running cost, so there is no (tf, tf) entry);
//   - J^T w and H v get a tf component summed over all nodes: every tile adds its owned
//     nodes in a fixed order and the last CTA adds the tile sums in tile order.
// The objective is the terminal (Mayer) cost sum_k mayer_k X_{N,k}; the final rows cover a
// subset of the state (X_{N,m} = mf for the rocket).
//
// Per node z = (r, v, m, u), with E = exp(-beta (r - 1)), D = Cd v^2 E / m:
//   f = (v,  -D - 1/r^2 + u Tmax / m,  -b Tmax u)
//   dv'/dr = beta D + 2/r^3,  dv'/dv = -2 Cd v E / m,  dv'/dm = (D - u Tmax / m) / m,
//   dv'/du = Tmax / m,  dm'/du = -b Tmax
//   d2v'/dr2 = -beta^2 D - 6/r^4,  d2v'/dv dr = -beta dv'/dv,  d2v'/dv2 = -2 Cd E / m,
//   d2v'/dm dr = -beta D / m,  d2v'/dm dv = -(dv'/dv) / m,  d2v'/dm2 = 2 (u Tmax / m - D) / m^2,
//   d2v'/du dm = -Tmax / m^2.
// Parameter derivatives (p = (Cd, beta, Tmax, b)), for (dc/dp)^T w next to J^T w:
//   dv'/dCd = -v^2 E / m,  dv'/dbeta = (r - 1) D,  dv'/dTmax = u / m,
//   dm'/dTmax = -b u,  dm'/db = -Tmax u.
//
// Work decomposition as for the other node models: a CTA of GT threads evaluates GT
// consecutive nodes and owns the first GT-1 (consecutive tiles overlap by one node), the
// Jacobian rows of a tile are staged in shared memory in their final order and stored with
// consecutive threads on consecutive addresses, and the right node of a defect row comes from
// lane+1 by shuffle (or the next warp's lane 0 through shared memory).  No atomics on values.
#include <cstring>

#include "exp_table.cuh"
#include "node_kernels.cuh"
#include "ocp_internal.h"

namespace ocpg {

constexpr int GT = 256;  // threads (= nodes) per CTA; a tile owns GT-1 nodes and rows

struct GodArgs {
  const double* __restrict__ x;
  const double* __restrict__ y;
  const double* __restrict__ vn;   // direction of J v and H v (length n)
  const double* __restrict__ vm;   // direction of J^T w (length m)
  double *f, *c, *g, *jv, *hv;
  double *ojv, *ojtv, *ohv;        // products
  double* partials;                // tile sums: tf components of J^T w and H v, then (dc/dp)^T w
  unsigned* counter;
  const double* p_dev;             // G_PAR: (Cd, beta, Tmax, b) read from the device
  double* dpar;                    // G_DP: (dc/dp)^T w, 4 doubles
  int64_t N, nb, uoff, tau, ntiles;  // tau: index of tf in x (n - 1)
  int64_t jbase[3];                  // first slot of the defect rows of each component
  int64_t hbase_u, hbase_t;          // Hessian slots: U block, tf row
  int hu, hpos_um;                   // U block entries per node; position of (u, m) in it
  double hh_fixed;                   // h / 2 of a fixed horizon
  double kappa;                      // 1 / (2N)
  double Cd, beta, Tmax, b, bT;      // bT = b Tmax
  double mayer[3];
  int finpos[3];                     // row of X_{N,k} among the final rows, or -1
  double one, mz;                    // 1.0 and -0.0 at run time (sums and products as FMAs)
};

// a + b, a - b, a * b issued as FMAs (same rounding; see fadd in models.cuh)
__device__ __forceinline__ double gadd(const GodArgs& a, double p, double q) { return fma(p, a.one, q); }
__device__ __forceinline__ double gsub(const GodArgs& a, double p, double q) { return fma(-q, a.one, p); }
__device__ __forceinline__ double gmul(const GodArgs& a, double p, double q) { return fma(p, q, a.mz); }

// Variant bits of k_god beside the outputs: G_DP adds (dc/dp)^T w to J^T w, G_PAR reads the
// parameters from the device.
constexpr unsigned G_DP = 1u << 10, G_PAR = 1u << 11;

// Last CTA to finish adds each series q < COUNT of tile sums, partials[q * ntiles + tile], in
// tile order (see finish_tiles) into dst[q] (skipped where null).
template <int COUNT>
__device__ __forceinline__ void finish_sums(const double* partials, int64_t ntiles, unsigned* counter,
                                            double* const (&dst)[COUNT], double* red) {
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
    if (!dst[q]) continue;  // CTA-uniform
    double sq = 0.0;
    for (int64_t i = threadIdx.x; i < ntiles; i += GT) sq = sq + __ldcg(partials + q * ntiles + i);
    sq = cta_sum<GT>(sq, red);
    if (threadIdx.x == 0) *dst[q] = sq;
  }
  if (threadIdx.x == 0) *counter = 0u;
}

template <unsigned OUT, bool FREE>
__global__ void __launch_bounds__(GT) k_god(const __grid_constant__ GodArgs a) {
  constexpr bool WF = OUT & O_F, WC = OUT & O_C, WG = OUT & O_G, WJ = OUT & O_J, WH = OUT & O_H;
  constexpr bool WJV = OUT & O_JV, WJTV = OUT & O_JTV, WHV = OUT & O_HV;
  constexpr bool NEEDD = WJ || WH || WJV || WJTV || WHV;   // first derivatives of f
  constexpr bool RED = FREE && (WJTV || WHV);              // tf components of the products
  constexpr bool DP = WJTV && (OUT & G_DP);                // (dc/dp)^T w
  constexpr bool PAR = OUT & G_PAR;
  constexpr int F1 = FREE ? 1 : 0;
  constexpr int CR = 4 + F1, CV = 8 + F1, CM = 4 + F1;     // entries per defect row of r, v, m
  constexpr int R = GT - 1;
  constexpr int OV = CR * R, OM = (CR + CV) * R;           // staged rows of v and m
  constexpr int EW = GT / 32 + 1;
  extern __shared__ __align__(16) double sm[];
  __shared__ double sEdge[9 * EW];                         // lane-0 values of pb, jA, fk per warp
  __shared__ double red0[GT], red1[GT];
  // the full kernel also serves output subsets: NULL outputs are neither computed nor stored
  const bool sF = WF && a.f, sC = WC && a.c, sG = WG && a.g, sJ = WJ && a.jv, sH = WH && a.hv;
  const bool doH = sH || WHV;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t N = a.N;
  __shared__ double sHH;
  double hh = a.hh_fixed;
  if (FREE) {  // hh = tf / (2N): one division per CTA (a per-thread division costs every node)
    if (t == 0) sHH = (__ldg(a.x + a.tau) / (double)N) * 0.5;
    __syncthreads();
    hh = sHH;
  }
  const double mhh = -hh, mk = -a.kappa;
  // the parameters: kernel arguments, or device memory with PAR (bT = b Tmax as on the host)
  const double Cd = PAR ? __ldg(a.p_dev) : a.Cd, beta = PAR ? __ldg(a.p_dev + 1) : a.beta;
  const double Tmax = PAR ? __ldg(a.p_dev + 2) : a.Tmax, bpar = PAR ? __ldg(a.p_dev + 3) : a.b;
  const double bT = PAR ? gmul(a, bpar, Tmax) : a.bT;
  double vt = 0.0;  // tf component of the direction
  if (FREE && (WJV || WHV)) vt = __ldg(a.vn + a.tau);

  for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * R;
    const int64_t own_end = min(r0 + R, N + 1);
    const int64_t row_end = min(own_end, N);
    const int nown = (int)(own_end - r0);
    const int nrows = (int)max(row_end - r0, (int64_t)0);
    const int64_t j = r0 + t;
    const bool act = j <= row_end;
    const bool own = t < nown;
    // the tile holds node 0 or node N (CTA-uniform): boundary-only FP64 work sits behind this
    // branch, since predicated-off FP64 instructions still take pipe slots in every warp
    const bool bnd = (r0 == 0) || (own_end == N + 1);
    double pa[3] = {0.0, 0.0, 0.0}, pb[3] = {0.0, 0.0, 0.0};
    double jA[3] = {0.0, 0.0, 0.0}, jB[3] = {0.0, 0.0, 0.0}, fk[3] = {0.0, 0.0, 0.0};
    double accJ = 0.0, accH = 0.0;
    double accP[4] = {0.0, 0.0, 0.0, 0.0};
    if (act) {
      const double r = __ldg(a.x + 3 * j), v = __ldg(a.x + 3 * j + 1), m = __ldg(a.x + 3 * j + 2);
      const double u = __ldg(a.x + a.uoff + j);
      const double E = exp_tab(fma(-beta, r, beta), a.one, a.mz);  // exp(-beta (r - 1))
      const double im = recip(a.one, m), ir = recip(a.one, r);
      const double ir2 = gmul(a, ir, ir);
      const double q1 = gmul(a, gmul(a, Cd, E), im);        // Cd E / m
      const double D = gmul(a, gmul(a, q1, v), v);
      const double aU = gmul(a, Tmax, im);                  // dv'/du = Tmax / m
      const double fv = fma(u, aU, -gadd(a, D, ir2));
      const double fm = gmul(a, -bT, u);
      pa[0] = fma(hh, v, r);  pb[0] = fma(mhh, v, r);
      pa[1] = fma(hh, fv, v); pb[1] = fma(mhh, fv, v);
      pa[2] = fma(hh, fm, m); pb[2] = fma(mhh, fm, m);
      if (FREE && (WJ || WJV || WJTV)) {
        fk[0] = gmul(a, mk, v);
        fk[1] = gmul(a, mk, fv);
        fk[2] = gmul(a, mk, fm);
      }
      if (NEEDD) {
        const double ar = fma(beta, D, gmul(a, 2.0, gmul(a, ir2, ir)));   // beta D + 2/r^3
        const double av = gmul(a, -2.0, gmul(a, q1, v));                     // -2 Cd v E / m
        const double am = gmul(a, gsub(a, D, gmul(a, u, aU)), im);          // (D - u Tmax/m) / m
        // Jacobian values without the identity: -hh df/dz
        const double jr = gmul(a, mhh, ar), jvv = gmul(a, mhh, av), jm = gmul(a, mhh, am);
        const double ju = gmul(a, mhh, aU), jmu = gmul(a, hh, bT);
        if (sJ) {  // left part of row t, right part of row t-1
          if (t < nrows) {
            double* rr = sm + t * CR;
            double* rv = sm + OV + t * CV;
            double* rm = sm + OM + t * CM;
            rr[0] = -1.0; rr[1] = mhh;
            rv[0] = jr; rv[1] = fma(jvv, a.one, -1.0); rv[2] = jm; rv[6] = ju;
            rm[0] = -1.0; rm[2] = jmu;
          }
          if (t >= 1 && t - 1 < nrows) {
            double* rr = sm + (t - 1) * CR;
            double* rv = sm + OV + (t - 1) * CV;
            double* rm = sm + OM + (t - 1) * CM;
            rr[2] = 1.0; rr[3] = mhh;
            rv[3] = jr; rv[4] = fma(jvv, a.one, 1.0); rv[5] = jm; rv[7] = ju;
            rm[1] = 1.0; rm[3] = jmu;
          }
        }
        double vz[4] = {0.0, 0.0, 0.0, 0.0};
        if (WJV || WHV) {
          vz[0] = __ldg(a.vn + 3 * j); vz[1] = __ldg(a.vn + 3 * j + 1); vz[2] = __ldg(a.vn + 3 * j + 2);
          vz[3] = __ldg(a.vn + a.uoff + j);
        }
        if (WJV) {  // node shares of rows (k, j-1) and (k, j): p_k +- v_{X_j,k}
          double p0 = gmul(a, mhh, vz[1]);
          double p1 = fma(jr, vz[0], fma(jvv, vz[1], fma(jm, vz[2], gmul(a, ju, vz[3]))));
          double p2 = gmul(a, jmu, vz[3]);
          if (FREE) { p0 = fma(fk[0], vt, p0); p1 = fma(fk[1], vt, p1); p2 = fma(fk[2], vt, p2); }
          const double p[3] = {p0, p1, p2};
#pragma unroll
          for (int k = 0; k < 3; ++k) { jA[k] = gadd(a, p[k], vz[k]); jB[k] = gsub(a, p[k], vz[k]); }
          if (own && j == 0) {
#pragma unroll
            for (int k = 0; k < 3; ++k) a.ojv[k] = vz[k];
          }
          if (own && j == N) {
#pragma unroll
            for (int k = 0; k < 3; ++k)
              if (a.finpos[k] >= 0) a.ojv[3 + a.finpos[k]] = vz[k];
          }
        }
        if (WJTV && own) {
          double wl[3], wr[3], wb[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const double* row = a.vm + a.nb + (int64_t)k * N;
            wl[k] = (j >= 1) ? __ldg(row + j - 1) : 0.0;
            wr[k] = (j < N) ? __ldg(row + j) : 0.0;
            wb[k] = gadd(a, wl[k], wr[k]);
          }
          double o[4];
          o[0] = fma(wb[1], jr, gsub(a, wl[0], wr[0]));
          o[1] = fma(wb[1], jvv, fma(wb[0], mhh, gsub(a, wl[1], wr[1])));
          o[2] = fma(wb[1], jm, gsub(a, wl[2], wr[2]));
          o[3] = fma(wb[2], jmu, gmul(a, wb[1], ju));
          if (bnd) {
            if (j == 0) {
#pragma unroll
              for (int k = 0; k < 3; ++k) o[k] = gadd(a, o[k], __ldg(a.vm + k));
            }
            if (j == N) {
#pragma unroll
              for (int k = 0; k < 3; ++k)
                if (a.finpos[k] >= 0) o[k] = gadd(a, o[k], __ldg(a.vm + 3 + a.finpos[k]));
            }
          }
          a.ojtv[3 * j] = o[0]; a.ojtv[3 * j + 1] = o[1]; a.ojtv[3 * j + 2] = o[2];
          a.ojtv[a.uoff + j] = o[3];
          if (FREE) accJ = fma(wb[0], fk[0], fma(wb[1], fk[1], gmul(a, wb[2], fk[2])));
          if (DP) {  // sum_k wbar_k (-hh df_k/dp_i)
            const double vEm = gmul(a, gmul(a, gmul(a, E, im), v), v);        // v^2 E / m
            accP[0] = gmul(a, wb[1], gmul(a, hh, vEm));
            accP[1] = gmul(a, wb[1], gmul(a, mhh, gmul(a, D, gsub(a, r, a.one))));
            accP[2] = fma(wb[1], gmul(a, mhh, gmul(a, u, im)), gmul(a, wb[2], gmul(a, hh, gmul(a, bpar, u))));
            accP[3] = gmul(a, wb[2], gmul(a, hh, gmul(a, Tmax, u)));
          }
        }
        if (doH && own) {
          // multiplier sums ybar_k = y_{k,j-1} + y_{k,j} (v always; r and m for the tf row)
          double yb[3] = {0.0, 0.0, 0.0};
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            if (k == 1 || FREE) {
              const double* row = a.y + a.nb + (int64_t)k * N;
              const double yl = (j >= 1) ? __ldg(row + j - 1) : 0.0;
              const double yr = (j < N) ? __ldg(row + j) : 0.0;
              yb[k] = gadd(a, yl, yr);
            }
          }
          const double y1 = gmul(a, mhh, yb[1]);
          const double ir4 = gmul(a, ir2, ir2);
          double hd[7];
          hd[0] = gmul(a, y1, fma(-gmul(a, beta, beta), D, gmul(a, -6.0, ir4)));   // (r, r)
          hd[1] = gmul(a, y1, gmul(a, -beta, av));                                 // (v, r)
          hd[2] = gmul(a, y1, gmul(a, -2.0, q1));                                    // (v, v)
          hd[3] = gmul(a, y1, gmul(a, gmul(a, -beta, D), im));                     // (m, r)
          hd[4] = gmul(a, y1, gmul(a, -av, im));                                     // (m, v)
          hd[5] = gmul(a, y1, gmul(a, gmul(a, 2.0, gsub(a, gmul(a, u, aU), D)), gmul(a, im, im)));  // (m, m)
          hd[6] = gmul(a, y1, gmul(a, -aU, im));                                     // (u, m)
          double tr = 0.0, tv = 0.0, tm = 0.0, tu = 0.0;  // tf row: -kappa sum_k ybar_k df_k/dz
          if (FREE) {
            tr = gmul(a, mk, gmul(a, yb[1], ar));
            tv = gmul(a, mk, fma(yb[1], av, yb[0]));
            tm = gmul(a, mk, gmul(a, yb[1], am));
            tu = gmul(a, mk, fma(yb[1], aU, gmul(a, -bT, yb[2])));
          }
          if (sH) {
#pragma unroll
            for (int e = 0; e < 6; ++e) a.hv[6 * j + e] = hd[e];
            // U block: (u, m), and (u, u) when a path inequality needs it (zero here; the path
            // rows add their part)
            for (int e = 0; e < a.hu; ++e) a.hv[a.hbase_u + (int64_t)a.hu * j + e] = (e == a.hpos_um) ? hd[6] : 0.0;
            if (FREE) {
              a.hv[a.hbase_t + 3 * j] = tr;
              a.hv[a.hbase_t + 3 * j + 1] = tv;
              a.hv[a.hbase_t + 3 * j + 2] = tm;
              a.hv[a.hbase_t + 3 * (N + 1) + j] = tu;
            }
          }
          if (WHV) {
            double o[4];
            o[0] = fma(hd[0], vz[0], fma(hd[1], vz[1], gmul(a, hd[3], vz[2])));
            o[1] = fma(hd[1], vz[0], fma(hd[2], vz[1], gmul(a, hd[4], vz[2])));
            o[2] = fma(hd[3], vz[0], fma(hd[4], vz[1], fma(hd[5], vz[2], gmul(a, hd[6], vz[3]))));
            o[3] = gmul(a, hd[6], vz[2]);
            if (FREE) {
              o[0] = fma(tr, vt, o[0]); o[1] = fma(tv, vt, o[1]); o[2] = fma(tm, vt, o[2]); o[3] = fma(tu, vt, o[3]);
              accH = fma(tr, vz[0], fma(tv, vz[1], fma(tm, vz[2], gmul(a, tu, vz[3]))));
            }
            a.ohv[3 * j] = o[0]; a.ohv[3 * j + 1] = o[1]; a.ohv[3 * j + 2] = o[2];
            a.ohv[a.uoff + j] = o[3];
          }
        }
      }
      if (own) {
        const double zx[3] = {r, v, m};
        if (sG) {  // the terminal cost is the only objective term
#pragma unroll
          for (int k = 0; k < 3; ++k) a.g[3 * j + k] = (j == N) ? a.mayer[k] : 0.0;
          a.g[a.uoff + j] = 0.0;
          if (FREE && j == 0) a.g[a.tau] = 0.0;
        }
        if (sF && bnd && j == N) *a.f = fma(a.mayer[0], r, fma(a.mayer[1], v, gmul(a, a.mayer[2], m)));
        if (j == 0) {
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            if (sC) a.c[k] = zx[k];
            if (sJ) a.jv[k] = 1.0;
          }
        }
        if (j == N) {
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            if (a.finpos[k] < 0) continue;
            if (sC) a.c[3 + a.finpos[k]] = zx[k];
            if (sJ) a.jv[3 + a.finpos[k]] = 1.0;
          }
        }
      }
    }
    // ---- defect rows: the right node's share comes from lane+1 (or the next warp's lane 0)
    double nbp[3], nbA[3], nbF[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (WC) {
        nbp[k] = __shfl_down_sync(0xffffffffu, pb[k], 1);
        if (lane == 0) sEdge[warp * 3 + k] = pb[k];
      }
      if (WJV) {
        nbA[k] = __shfl_down_sync(0xffffffffu, jA[k], 1);
        if (lane == 0) sEdge[3 * EW + warp * 3 + k] = jA[k];
      }
      if (FREE && WJ) {
        nbF[k] = __shfl_down_sync(0xffffffffu, fk[k], 1);
        if (lane == 0) sEdge[6 * EW + warp * 3 + k] = fk[k];
      }
    }
    if (WC || WJ || WJV) __syncthreads();
    if (t < nrows) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int64_t row = a.nb + (int64_t)k * N + j;
        if (sC) {
          const double right = (lane == 31) ? sEdge[(warp + 1) * 3 + k] : nbp[k];
          a.c[row] = gsub(a, right, pa[k]);
        }
        if (WJV) {
          const double right = (lane == 31) ? sEdge[3 * EW + (warp + 1) * 3 + k] : nbA[k];
          a.ojv[row] = gadd(a, jB[k], right);
        }
        if (FREE && WJ && sJ) {  // the tf entry closes the row
          const double right = (lane == 31) ? sEdge[6 * EW + (warp + 1) * 3 + k] : nbF[k];
          const int off = (k == 0) ? t * CR + CR - 1 : (k == 1) ? OV + t * CV + CV - 1 : OM + t * CM + CM - 1;
          sm[off] = gadd(a, fk[k], right);
        }
      }
    }
    if (FREE && WJ) __syncthreads();
    // ---- copy-out of the staged Jacobian rows, coalesced (with the free final time every row
    // holds an odd number of entries, so a tile's range alternates its 16-byte phase)
    if (sJ) {
      const int cnt[3] = {CR, CV, CM};
      const int soff[3] = {0, OV, OM};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double* src = sm + soff[k];
        double* dst = a.jv + a.jbase[k] + r0 * cnt[k];
        const int total = nrows * cnt[k];
        for (int i = t; i < total; i += GT) dst[i] = src[i];
      }
    }
    if (RED) {
      const double s0 = tile_sum<GT>(accJ, red0, a.one);
      const double s1 = tile_sum<GT>(accH, red1, a.one);
      if (t == 0) {
        a.partials[tile] = s0;
        a.partials[a.ntiles + tile] = s1;
      }
    }
    __syncthreads();
    if (DP) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const double si = tile_sum<GT>(accP[i], red0, a.one);
        if (t == 0) a.partials[(2 + i) * a.ntiles + tile] = si;
        __syncthreads();
      }
    }
  }
  if (RED || DP) {
    double* const dst[6] = {(RED && WJTV) ? a.ojtv + a.tau : nullptr, (RED && WHV) ? a.ohv + a.tau : nullptr,
                            DP ? a.dpar : nullptr, DP ? a.dpar + 1 : nullptr, DP ? a.dpar + 2 : nullptr,
                            DP ? a.dpar + 3 : nullptr};
    finish_sums<6>(a.partials, a.ntiles, a.counter, dst, red0);
  }
}

// ======================================================================================
// Host side
// ======================================================================================
static void fill_god(const ocp* h, GodArgs& a) {
  memset(&a, 0, sizeof(a));
  const Pattern& P = h->pat;
  a.N = h->N;
  a.nb = P.nb;
  a.uoff = 3 * (h->N + 1);
  a.tau = P.free_tf ? P.n - 1 : -1;
  a.ntiles = (h->N + 1 + GT - 2) / (GT - 1);
  for (int k = 0; k < 3; ++k) a.jbase[k] = P.jbase[k];
  a.hbase_u = P.hbase_u;
  a.hbase_t = P.hbase_t;
  a.hu = P.hu;
  a.hpos_um = 0;
  for (int e = 0; e < P.hu; ++e)
    if (P.hent[P.hx + e].first == 3 && P.hent[P.hx + e].second == 2) a.hpos_um = e;
  a.hh_fixed = h->hh;
  a.kappa = 1.0 / (2.0 * (double)h->N);
  a.Cd = h->params[0];
  a.beta = h->params[1];
  a.Tmax = h->params[2];
  a.b = h->params[3];
  a.bT = h->params[3] * h->params[2];
  a.p_dev = h->p0_dev;
  for (int k = 0; k < 3; ++k) a.mayer[k] = h->mayer.empty() ? 0.0 : h->mayer[k];
  for (int k = 0; k < 3; ++k) a.finpos[k] = -1;
  for (size_t i = 0; i < P.fin.size(); ++i) a.finpos[P.fin[i]] = (int)i;
  a.one = 1.0;
  a.mz = -0.0;
  a.partials = h->d_partials;
  a.counter = h->d_counter;
}

template <unsigned OUT, bool FREE>
static cudaError_t god_launch(const GodArgs& a, cudaStream_t s) {
  constexpr int F1 = FREE ? 1 : 0;
  const size_t smem = (OUT & O_J) ? sizeof(double) * (size_t)(16 + 3 * F1) * (GT - 1) : 0;
  const int grid = (int)(a.ntiles < 0x7fffffff ? a.ntiles : 0x7fffffff);
  k_god<OUT, FREE><<<grid, GT, smem, s>>>(a);  // (G_DP, G_PAR bits in OUT)
  return cudaGetLastError();
}

template <unsigned OUT>
static cudaError_t god_launch_tf(const ocp* h, const GodArgs& a, cudaStream_t s) {
  return h->pat.free_tf ? god_launch<OUT, true>(a, s) : god_launch<OUT, false>(a, s);
}

ocp_status goddard_eval(ocp* h, unsigned out, const EvalCall& c, cudaStream_t s) {
  if (c.range || c.B != 0 || c.E != h->N + 1)
    return set_err(h, OCP_EMODEL, "node ranges are not provided for the Goddard model");
  GodArgs a;
  fill_god(h, a);
  if (2 * a.ntiles > h->max_partials) return set_err(h, OCP_EDIM, "too many tiles for the reduction scratch");
  a.x = c.x; a.y = c.y; a.f = c.f; a.c = c.c; a.g = c.g; a.jv = c.jv; a.hv = c.hv;
  a.vn = c.vn; a.vm = c.vm; a.ojv = c.ojv; a.ojtv = c.ojtv; a.ohv = c.ohv;
  cudaError_t e;
  if (a.p_dev) {  // device parameters: the constraints alone
    if (out != O_C) return set_err(h, OCP_EMODEL, "device parameters: the constraints only");
    return cuda_err(h, god_launch_tf<O_ALL | G_PAR>(h, a, s), "Goddard kernel launch");
  }
  switch (out) {
    case O_STEP: e = god_launch_tf<O_STEP>(h, a, s); break;
    case O_J | O_H: e = god_launch_tf<O_J | O_H>(h, a, s); break;
    default: e = god_launch_tf<O_ALL>(h, a, s); break;  // subsets: NULL outputs are skipped
  }
  return cuda_err(h, e, "Goddard kernel launch");
}

ocp_status goddard_prod(ocp* h, const ProdCall& c, cudaStream_t s) {
  GodArgs a;
  fill_god(h, a);
  if (2 * a.ntiles > h->max_partials) return set_err(h, OCP_EDIM, "too many tiles for the reduction scratch");
  if (c.kind == P_JTPROD && (c.B != 0 || (c.E >= 0 && c.E != h->N + 1)))
    return set_err(h, OCP_EMODEL, "node ranges are not provided for the Goddard model");
  a.x = c.x;
  cudaError_t e;
  const bool par = a.p_dev != nullptr;  // device-resident parameters
  if (c.kind == P_JPROD) {
    a.vn = c.v; a.ojv = c.out;
    e = par ? god_launch_tf<O_JV | G_PAR>(h, a, s) : god_launch_tf<O_JV>(h, a, s);
  } else if (c.kind == P_JTPROD) {
    a.vm = c.v; a.ojtv = c.out; a.dpar = c.dmu;
    if (c.dmu && 6 * a.ntiles > h->max_partials) return set_err(h, OCP_EDIM, "too many tiles for the reduction scratch");
    if (!c.dmu) e = par ? god_launch_tf<O_JTV | G_PAR>(h, a, s) : god_launch_tf<O_JTV>(h, a, s);
    else e = par ? god_launch_tf<O_JTV | G_DP | G_PAR>(h, a, s) : god_launch_tf<O_JTV | G_DP>(h, a, s);
  } else {
    a.y = c.y; a.vn = c.v; a.ohv = c.out;
    e = par ? god_launch_tf<O_HV | G_PAR>(h, a, s) : god_launch_tf<O_HV>(h, a, s);
  }
  return cuda_err(h, e, "Goddard product launch");
}

}  // namespace ocpg
