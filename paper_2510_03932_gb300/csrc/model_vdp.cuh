// Device model of the Van der Pol dynamics (the conventions of every model are stated in
// model_base.cuh).
#pragma once
#include "model_base.cuh"

namespace ocpg {

// ------------------------------------------------------------------------------------
// Van der Pol:  f0 = x2,  f1 = mu (1 - x1^2) x2 - x1 + u.
//   df1/dx1 = -2 mu x1 x2 - 1,  df1/dx2 = mu (1 - x1^2),  df1/du = 1
//   d2f1/dx1^2 = -2 mu x2,  d2f1/dx1dx2 = -2 mu x1
//   df1/dmu = (1 - x1^2) x2,  d2f1/dmu dx1 = -2 x1 x2,  d2f1/dmu dx2 = 1 - x1^2
// Constants: c[0] = 2 hh mu, c[1] = hh mu, c[2] = -hh mu.
// ------------------------------------------------------------------------------------
struct VdP {
  static constexpr int EVAL_MIN_CTAS = 0;
  static constexpr int NX = 2, NU = 1, NZ = 3;
  static constexpr int MAXRX = 2, MAXRU = 1;
  OCP_TABLE1(RX, int, NX, {2, 2})
  OCP_TABLE1(RU, int, NX, {0, 1})
  OCP_TABLE2(XV, int, NX, MAXRX, {{0, 1}, {0, 1}})
  OCP_TABLE2(UV, int, NX, MAXRU, {{-1}, {0}})
  OCP_TABLE2(JZ, bool, NX, MAXRX, {{true, false}, {false, false}})
  OCP_TABLE1(HK, bool, NX, {false, true})
  static constexpr int NHD = 2;
  OCP_TABLE1(HA, int, NHD, {0, 1})
  OCP_TABLE1(HB, int, NHD, {0, 0})
  static constexpr bool HAS_DPARAM = true;
  static constexpr int NP = 1;  // mu
  static constexpr bool FUSED_DP = false;  // dparams separately (cheap)
  OCP_TABLE2(DP, bool, NX, NP, {{false}, {true}})

  static void host_consts(const double* p, double hh, ModelConst& mc) {
    mc.hh = hh;
    mc.mhh = -hh;
    mc.one = 1.0;
    mc.mz = -0.0;
    mc.c[0] = 2.0 * hh * p[0];
    mc.c[1] = hh * p[0];
    mc.c[2] = -(hh * p[0]);
  }
  // Override of the parameter from a device scalar: constants as above.
  __device__ __forceinline__ static void device_param(ModelConst& K, double mu) {
    K.c[0] = (2.0 * K.hh) * mu;
    K.c[1] = K.hh * mu;
    K.c[2] = -K.c[1];
  }
  __device__ __forceinline__ static void device_params(ModelConst& K, const double* p) { device_param(K, __ldg(p)); }

  template <bool WC, bool WJ, bool WH>
  __device__ __forceinline__ static void eval(const ModelConst& K, const double (&z)[NZ], const double (&yb)[NX],
                                              const double (&cqd)[NZ], double (&pa)[NX], double (&pb)[NX],
                                              double (&mjx)[NX][MAXRX], double (&mju)[NX][MAXRU],
                                              double (&hd)[NHD]) {
    const double x1 = z[0], x2 = z[1], u = z[2];
    if (WJ || WC) {
      // m12 = -hh df1/dx2 = hh mu (x1^2 - 1)
      const double a = fmul(K, K.c[1], x1);
      const double m12 = fma(a, x1, K.c[2]);
      if (WJ) {
        mjx[0][0] = 0.0;                              // x1 in row 0: identity only
        mjx[0][1] = K.mhh;                            // x2 in row 0: -hh * 1
        mjx[1][0] = fma(K.c[0], fmul(K, x1, x2), K.hh);  // -hh (-2 mu x1 x2 - 1)
        mjx[1][1] = m12;
        mju[1][0] = K.mhh;
      }
      if (WC) {
        pa[0] = fma(K.hh, x2, x1);
        pb[0] = fma(K.mhh, x2, x1);
        // hh f1 = -m12 x2 + hh (u - x1)
        const double d = fsub(K, u, x1);
        pa[1] = fma(-m12, x2, fma(K.hh, d, x2));
        pb[1] = fma(m12, x2, fma(K.mhh, d, x2));
      }
    }
    if (WH) {
      const double t = fmul(K, K.c[0], yb[1]);
      hd[0] = fma(t, x2, cqd[0]);   // (x1, x1)
      hd[1] = fmul(K, t, x1);       // (x2, x1)
    }
  }

  // -hh df_k/dmu
  __device__ __forceinline__ static void dparam(const ModelConst& K, const double (&z)[NZ], double (&mdp)[NX]) {
    const double x1 = z[0], x2 = z[1];
    mdp[0] = 0.0;
    mdp[1] = fmul(K, K.mhh, fmul(K, fma(-x1, x1, 1.0), x2));
  }
  __device__ __forceinline__ static void dparams(const ModelConst& K, const double (&z)[NZ], double (&mdp)[NX][NP]) {
    double t[NX];
    dparam(K, z, t);
    mdp[0][0] = t[0];
    mdp[1][0] = t[1];
  }
  // sum_k wbar_k (-hh d2 f_k / dmu dz_v) for every local v
  __device__ __forceinline__ static void dparam_grad(const ModelConst& K, const double (&z)[NZ],
                                                     const double (&wb)[NX], double (&out)[NZ]) {
    const double x1 = z[0], x2 = z[1];
    const double t = fmul(K, K.mhh, wb[1]);
    out[0] = fmul(K, fmul(K, -2.0, t), fmul(K, x1, x2));
    out[1] = fmul(K, t, fma(-x1, x1, 1.0));
    out[2] = 0.0;
  }
};

}  // namespace ocpg
