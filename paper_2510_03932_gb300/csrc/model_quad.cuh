// Device model of the quadrotor dynamics (the conventions of every model are stated in
// model_base.cuh).
#pragma once
#include "model_base.cuh"
#include "sincos_table.cuh"

namespace ocpg {

// ------------------------------------------------------------------------------------
// Quadrotor (the paper's second benchmark problem, appendix).  z = (x1..x9, u1..u4), local
// indices 0..12; x7, x8, x9 are the attitude angles, u1 the thrust per unit mass.
//   x1' = x2, x3' = x4, x5' = x6,
//   x2' = u1 P,  x4' = u1 Q,  x6' = u1 R - g,
//     P = c7 s8 c9 + s7 s9,  Q = c7 s8 s9 - s7 c9,  R = c7 c8     (ck = cos xk, sk = sin xk)
//   x7' = a e,  x8' = b,  x9' = a t + u4,
//     a = u2 c7 + u3 s7,  b = u3 c7 - u2 s7 (= da/dx7),  e = 1/c8,  t = s8 e (= tan x8).
// First derivatives (de/dx8 = e t, dt/dx8 = e^2):
//   P_7 = c7 s9 - s7 s8 c9,  P_8 = c7 c8 c9,  P_9 = s7 c9 - c7 s8 s9,
//   Q_7 = -(s7 s8 s9 + c7 c9),  Q_8 = c7 c8 s9,  Q_9 = P,   R_7 = -s7 c8,  R_8 = -c7 s8,
//   (a e)_7 = b e, (a e)_8 = a e t;  (b)_7 = -a;  (a t)_7 = b t, (a t)_8 = a e^2.
// Second derivatives of the three rotation rows (u1 enters linearly):
//   P_77 = P_99 = -P, P_78 = -s7 c8 c9, P_79 = -Q_7, P_88 = -c7 s8 c9, P_89 = -Q_8
//   Q_77 = Q_99 = -Q, Q_78 = -s7 c8 s9, Q_79 = P_7,  Q_88 = -c7 s8 s9, Q_89 = P_8
//   R_77 = R_88 = -R, R_78 = s7 s8
// and of the angle rows:  (a e)_77 = -a e, (a e)_78 = b e t, (a e)_88 = a e (t^2 + e^2),
//   (b)_77 = -b,  (a t)_77 = -a t, (a t)_78 = b e^2, (a t)_88 = 2 a e^2 t;  the mixed control
//   terms are the u2 / u3 coefficients of these.
// Hessian entries (a >= b): the lower triangle of {x7, x8, x9} and u1 x {x7, x8, x9} (rows
// x2', x4', x6'), u2 / u3 x {x7, x8} (rows x7', x8', x9').
// Constants: c[0] = g.
// ------------------------------------------------------------------------------------
struct Quadrotor {
  // 3 CTAs of 128 threads per SM (168 registers) for the evaluation kernels: measured faster than
  // the allocator's own choice (14% for the evaluation, 4% for the fused step, at 64-node tiles
  // and 6 CTAs) and than 4 CTAs (128 registers, larger spills: fused step 911 vs 832 us)
  static constexpr int EVAL_MIN_CTAS = 3;
  static constexpr int NX = 9, NU = 4, NZ = 13;
  static constexpr int MAXRX = 4, MAXRU = 3;
  OCP_TABLE1(RX, int, NX, {2, 4, 2, 4, 2, 3, 2, 2, 3})
  OCP_TABLE1(RU, int, NX, {0, 1, 0, 1, 0, 1, 2, 2, 3})
  OCP_TABLE2(XV, int, NX, MAXRX, {{0, 1, -1, -1}, {1, 6, 7, 8}, {2, 3, -1, -1}, {3, 6, 7, 8}, {4, 5, -1, -1},
                                  {5, 6, 7, -1}, {6, 7, -1, -1}, {6, 7, -1, -1}, {6, 7, 8, -1}})
  OCP_TABLE2(UV, int, NX, MAXRU, {{-1, -1, -1}, {0, -1, -1}, {-1, -1, -1}, {0, -1, -1}, {-1, -1, -1},
                                  {0, -1, -1}, {1, 2, -1}, {1, 2, -1}, {1, 2, 3}})
  OCP_TABLE2(JZ, bool, NX, MAXRX, {{true, false, false, false}, {true, false, false, false},
                                   {true, false, false, false}, {true, false, false, false},
                                   {true, false, false, false}, {true, false, false, false},
                                   {false, false, false, false}, {false, true, false, false},
                                   {false, false, true, false}})
  OCP_TABLE1(HK, bool, NX, {false, true, false, true, false, true, true, true, true})
  static constexpr int NHD = 13;
  OCP_TABLE1(HA, int, NHD, {6, 7, 7, 8, 8, 8, 9, 9, 9, 10, 10, 11, 11})
  OCP_TABLE1(HB, int, NHD, {6, 6, 7, 6, 7, 8, 6, 7, 8, 6, 7, 6, 7})
  static constexpr bool HAS_DPARAM = false;
  static constexpr int NP = 1;  // g
  static constexpr bool FUSED_DP = false;  // dparams separately (a constant)
  OCP_TABLE2(DP, bool, NX, NP, {{false}, {false}, {false}, {false}, {false}, {true}, {false}, {false}, {false}})

  static void host_consts(const double* p, double hh, ModelConst& mc) {
    mc.hh = hh;
    mc.mhh = -hh;
    mc.one = 1.0;
    mc.mz = -0.0;
    mc.c[0] = p[0];
  }
  __device__ __forceinline__ static void device_param(ModelConst&, double) {}
  __device__ __forceinline__ static void device_params(ModelConst& K, const double* p) { K.c[0] = __ldg(p); }

  template <bool WC, bool WJ, bool WH>
  __device__ __forceinline__ static void eval(const ModelConst& K, const double (&z)[NZ], const double (&yb)[NX],
                                              const double (&cqd)[NZ], double (&pa)[NX], double (&pb)[NX],
                                              double (&mjx)[NX][MAXRX], double (&mju)[NX][MAXRU],
                                              double (&hd)[NHD]) {
    const double hh = K.hh, mhh = K.mhh;
    const double u1 = z[9], u2 = z[10], u3 = z[11];
    double s7, c7, s8, c8, s9, c9;
    sincos_tab(K, z[6], s7, c7);
    sincos_tab(K, z[7], s8, c8);
    sincos_tab(K, z[8], s9, c9);
    const double e = recip(K.one, c8);
    const double t = fmul(K, s8, e);
    const double c7s8 = fmul(K, c7, s8), s7s8 = fmul(K, s7, s8);
    const double c7c8 = fmul(K, c7, c8), s7c8 = fmul(K, s7, c8);
    const double P = fma(c7s8, c9, fmul(K, s7, s9));
    const double Q = fma(c7s8, s9, fmul(K, -s7, c9));
    const double a = fma(u2, c7, fmul(K, u3, s7));
    const double b = fma(u3, c7, fmul(K, -u2, s7));
    const double ae = fmul(K, a, e);
    if (WC) {
      const double f[NX] = {z[1], fmul(K, u1, P), z[3], fmul(K, u1, Q), z[5], fma(u1, c7c8, -K.c[0]),
                            ae, b, fma(a, t, z[12])};
#pragma unroll
      for (int k = 0; k < NX; ++k) {
        pa[k] = fma(hh, f[k], z[k]);
        pb[k] = fma(mhh, f[k], z[k]);
      }
    }
    if (WJ || WH) {
      const double P7 = fma(c7, s9, fmul(K, -s7s8, c9));
      const double P8 = fmul(K, c7c8, c9);
      const double P9 = fma(s7, c9, fmul(K, -c7s8, s9));
      const double Q7 = -fma(s7s8, s9, fmul(K, c7, c9));
      const double Q8 = fmul(K, c7c8, s9);
      const double e2 = fmul(K, e, e);
      if (WJ) {
        const double mu1 = fmul(K, mhh, u1);
        mjx[0][0] = 0.0; mjx[0][1] = mhh;
        mjx[1][0] = 0.0; mjx[1][1] = fmul(K, mu1, P7); mjx[1][2] = fmul(K, mu1, P8); mjx[1][3] = fmul(K, mu1, P9);
        mju[1][0] = fmul(K, mhh, P);
        mjx[2][0] = 0.0; mjx[2][1] = mhh;
        mjx[3][0] = 0.0; mjx[3][1] = fmul(K, mu1, Q7); mjx[3][2] = fmul(K, mu1, Q8); mjx[3][3] = fmul(K, mu1, P);
        mju[3][0] = fmul(K, mhh, Q);
        mjx[4][0] = 0.0; mjx[4][1] = mhh;
        mjx[5][0] = 0.0; mjx[5][1] = fmul(K, -mu1, s7c8); mjx[5][2] = fmul(K, -mu1, c7s8);
        mju[5][0] = fmul(K, mhh, c7c8);
        const double mhe = fmul(K, mhh, e);
        mjx[6][0] = fmul(K, mhe, b); mjx[6][1] = fmul(K, fmul(K, mhh, ae), t);
        mju[6][0] = fmul(K, mhe, c7); mju[6][1] = fmul(K, mhe, s7);
        mjx[7][0] = fmul(K, hh, a); mjx[7][1] = 0.0;
        mju[7][0] = fmul(K, hh, s7); mju[7][1] = fmul(K, mhh, c7);
        const double mht = fmul(K, mhh, t);
        mjx[8][0] = fmul(K, mht, b); mjx[8][1] = fmul(K, fmul(K, mhh, a), e2); mjx[8][2] = 0.0;
        mju[8][0] = fmul(K, mht, c7); mju[8][1] = fmul(K, mht, s7); mju[8][2] = mhh;
      }
      if (WH) {
        // -hh ybar_k for the rows with a Hessian, and the u1-scaled ones of the rotation rows
        const double m1 = fmul(K, mhh, yb[1]), m3 = fmul(K, mhh, yb[3]), m5 = fmul(K, mhh, yb[5]);
        const double m6 = fmul(K, mhh, yb[6]), m7 = fmul(K, mhh, yb[7]), m8 = fmul(K, mhh, yb[8]);
        const double w1 = fmul(K, m1, u1), w3 = fmul(K, m3, u1), w5 = fmul(K, m5, u1);
        const double A1 = fma(m6, e, fmul(K, m8, t));      // coefficient of -a at (x7, x7) and of -s7 / c7
        const double B1 = fma(m6, t, fmul(K, m8, e));      // (x8, x7) and mixed x8 terms, times e
        const double C1 = fma(w1, c9, fmul(K, w3, s9));
        const double PQ = fma(w1, P, fmul(K, w3, Q));
        // (x7, x7)
        hd[0] = fsub(K, cqd[6], fma(w5, c7c8, fma(a, A1, fma(m7, b, PQ))));
        // (x8, x7)
        hd[1] = fma(fmul(K, b, e), B1, fma(w5, s7s8, fmul(K, -s7c8, C1)));
        // (x8, x8): a e (m6 (t^2 + e^2) + 2 m8 e t)
        const double q88 = fma(m6, fma(t, t, e2), fmul(K, fmul(K, 2.0, m8), fmul(K, e, t)));
        hd[2] = fma(ae, q88, fsub(K, cqd[7], fma(c7s8, C1, fmul(K, w5, c7c8))));
        // (x9, x7), (x9, x8), (x9, x9)
        hd[3] = fma(w3, P7, fmul(K, -w1, Q7));
        hd[4] = fma(w3, P8, fmul(K, -w1, Q8));
        hd[5] = fsub(K, cqd[8], PQ);
        // (u1, x7), (u1, x8), (u1, x9)
        hd[6] = fma(m1, P7, fma(m3, Q7, fmul(K, -m5, s7c8)));
        hd[7] = fma(m1, P8, fma(m3, Q8, fmul(K, -m5, c7s8)));
        hd[8] = fma(m1, P9, fmul(K, m3, P));
        // (u2, x7), (u2, x8), (u3, x7), (u3, x8)
        hd[9] = fma(-s7, A1, fmul(K, -m7, c7));
        hd[10] = fmul(K, fmul(K, c7, e), B1);
        hd[11] = fma(c7, A1, fmul(K, -m7, s7));
        hd[12] = fmul(K, fmul(K, s7, e), B1);
      }
    }
  }
  __device__ __forceinline__ static void dparam(const ModelConst&, const double (&)[NZ], double (&mdp)[NX]) {
    for (int k = 0; k < NX; ++k) mdp[k] = 0.0;
  }
  // -hh df_k/dg: only x6' = u1 R - g depends on g
  __device__ __forceinline__ static void dparams(const ModelConst& K, const double (&)[NZ], double (&mdp)[NX][NP]) {
#pragma unroll
    for (int k = 0; k < NX; ++k) mdp[k][0] = 0.0;
    mdp[5][0] = K.hh;
  }
  __device__ __forceinline__ static void dparam_grad(const ModelConst&, const double (&)[NZ], const double (&)[NX],
                                                     double (&out)[NZ]) {
    for (int v = 0; v < NZ; ++v) out[v] = 0.0;
  }
};

}  // namespace ocpg
