// Device model of the double integrator dynamics (the conventions of every model are stated in
// model_base.cuh).
#pragma once
#include "model_base.cuh"

namespace ocpg {

// ------------------------------------------------------------------------------------
// Double integrator (paper Sec. 5):  f0 = x2,  f1 = u.  Linear: no Hessian.
// ------------------------------------------------------------------------------------
struct Dint {
  static constexpr int EVAL_MIN_CTAS = 0;
  static constexpr int NX = 2, NU = 1, NZ = 3;
  static constexpr int MAXRX = 2, MAXRU = 1;
  OCP_TABLE1(RX, int, NX, {2, 1})
  OCP_TABLE1(RU, int, NX, {0, 1})
  OCP_TABLE2(XV, int, NX, MAXRX, {{0, 1}, {1, -1}})
  OCP_TABLE2(UV, int, NX, MAXRU, {{-1}, {0}})
  OCP_TABLE2(JZ, bool, NX, MAXRX, {{true, false}, {true, false}})
  OCP_TABLE1(HK, bool, NX, {false, false})
  static constexpr int NHD = 0;
  OCP_TABLE1(HA, int, 1, {0})
  OCP_TABLE1(HB, int, 1, {0})
  static constexpr bool HAS_DPARAM = false;
  static constexpr int NP = 0;  // no parameters
  static constexpr bool FUSED_DP = false;
  OCP_TABLE2(DP, bool, NX, 1, {{false}, {false}})

  static void host_consts(const double*, double hh, ModelConst& mc) {
    mc.hh = hh;
    mc.mhh = -hh;
    mc.one = 1.0;
    mc.mz = -0.0;
  }
  __device__ __forceinline__ static void device_param(ModelConst&, double) {}
  __device__ __forceinline__ static void device_params(ModelConst&, const double*) {}

  template <bool WC, bool WJ, bool WH>
  __device__ __forceinline__ static void eval(const ModelConst& K, const double (&z)[NZ], const double (&)[NX],
                                              const double (&)[NZ], double (&pa)[NX], double (&pb)[NX],
                                              double (&mjx)[NX][MAXRX], double (&mju)[NX][MAXRU], double (&)[1]) {
    if (WJ) {
      mjx[0][0] = 0.0;
      mjx[0][1] = K.mhh;
      mjx[1][0] = 0.0;
      mju[1][0] = K.mhh;
    }
    if (WC) {
      pa[0] = fma(K.hh, z[1], z[0]);
      pb[0] = fma(K.mhh, z[1], z[0]);
      pa[1] = fma(K.hh, z[2], z[1]);
      pb[1] = fma(K.mhh, z[2], z[1]);
    }
  }
  __device__ __forceinline__ static void dparam(const ModelConst&, const double (&)[NZ], double (&mdp)[NX]) {
    mdp[0] = 0.0; mdp[1] = 0.0;
  }
  __device__ __forceinline__ static void dparams(const ModelConst&, const double (&)[NZ], double (&mdp)[NX][1]) {
    mdp[0][0] = 0.0; mdp[1][0] = 0.0;
  }
  __device__ __forceinline__ static void dparam_grad(const ModelConst&, const double (&)[NZ], const double (&)[NX],
                                                     double (&out)[NZ]) {
    out[0] = out[1] = out[2] = 0.0;
  }
};

}  // namespace ocpg
