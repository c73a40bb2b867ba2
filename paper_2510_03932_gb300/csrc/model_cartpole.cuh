// Device model of the cart-pole dynamics (the conventions of every model are stated in
// model_base.cuh).
#pragma once
#include "model_base.cuh"
#include "sincos_table.cuh"

namespace ocpg {

// ------------------------------------------------------------------------------------
// Cart-pole, point-mass pole, theta from the downward vertical.  z = (p, pd, th, w, F).
//   D = mc + mp s^2,  A = F + mp s (l w^2 + g c),  B = -F c - s (mp l w^2 c + (mc+mp) g)
//   pdd = A / D,  thdd = B / (l D)
// Derivatives from  pdd D = A  and  thdd (l D) = B  differentiated in place (D depends on th
// only; D' = 2 mp s c, D'' = 2 mp (c^2 - s^2)):
//   pdd_t  = (A_t - pdd D') / D            A_t  = mp (l w^2 c + g (c^2 - s^2))
//   pdd_w  = A_w / D                       A_w  = 2 mp l w s
//   pdd_F  = 1 / D
//   pdd_tt = (A_tt - 2 pdd_t D' - pdd D'') / D     A_tt = -mp s (l w^2 + 4 g c)
//   pdd_tw = (A_tw - pdd_w D') / D                 A_tw = 2 mp l w c
//   pdd_ww = 2 mp l s / D,   pdd_tF = -pdd_F D' / D
//   thdd_t  = (B_t / l - thdd D') / D      B_t = F s - mp l w^2 (c^2 - s^2) - (mc+mp) g c
//   thdd_w  = B_w / (l D)                  B_w = -2 mp l w c s
//   thdd_F  = -c / (l D)
//   thdd_tt = (B_tt / l - 2 thdd_t D' - thdd D'') / D   B_tt = F c + 4 mp l w^2 s c + (mc+mp) g s
//   thdd_tw = (B_tw / l - thdd_w D') / D                B_tw = -2 mp l w (c^2 - s^2)
//   thdd_ww = -2 mp c s / D,   thdd_tF = (s / l - thdd_F D') / D
// Constants: c[0]=mc, c[1]=mp, c[2]=l, c[3]=g, c[4]=(mc+mp) g, c[5]=1/l, c[6]=mp l, c[7]=2 mp,
//            c[8]=mp g, c[9]=2 mp l, c[10]=4 g, c[11]=hh/l, c[12]=-hh/l, c[13]=3 mp l, c[14]=mc+mp.
// The kernels carry the angular acceleration scaled by l, Bu = B / D = l thdd, and its
// derivatives (Bu_t = (B_t - Bu D') / D, Bu_w = B_w / D, Bu_F = -c / D): the 1/l then enters
// only through the constants hh/l (defects, Jacobian) and the multiplier of the Hessian terms.
// ------------------------------------------------------------------------------------
struct CartPole {
  static constexpr int EVAL_MIN_CTAS = 0;
  static constexpr int NX = 4, NU = 1, NZ = 5;
  static constexpr int MAXRX = 3, MAXRU = 1;
  OCP_TABLE1(RX, int, NX, {2, 3, 2, 2})
  OCP_TABLE1(RU, int, NX, {0, 1, 0, 1})
  OCP_TABLE2(XV, int, NX, MAXRX, {{0, 1, -1}, {1, 2, 3}, {2, 3, -1}, {2, 3, -1}})
  OCP_TABLE2(UV, int, NX, MAXRU, {{-1}, {0}, {-1}, {0}})
  OCP_TABLE2(JZ, bool, NX, MAXRX, {{true, false, false}, {true, false, false}, {true, false, false},
                                   {false, false, false}})
  OCP_TABLE1(HK, bool, NX, {false, true, false, true})
  static constexpr int NHD = 4;
  OCP_TABLE1(HA, int, NHD, {2, 3, 3, 4})
  OCP_TABLE1(HB, int, NHD, {2, 2, 3, 2})
  static constexpr bool HAS_DPARAM = false;
  static constexpr int NP = 4;  // (mc, mp, l, g)
  OCP_TABLE2(DP, bool, NX, NP, {{false, false, false, false}, {true, true, true, true},
                                {false, false, false, false}, {true, true, true, true}})

  // The parameter-dependent constants (the same arithmetic on the host and on the device).
  __host__ __device__ static void param_consts(const double* p, double hh, ModelConst& mc) {
    const double m_c = p[0], m_p = p[1], l = p[2], g = p[3];
    mc.c[0] = m_c; mc.c[1] = m_p; mc.c[2] = l; mc.c[3] = g;
    mc.c[4] = (m_c + m_p) * g; mc.c[5] = 1.0 / l; mc.c[6] = m_p * l; mc.c[7] = 2.0 * m_p;
    mc.c[8] = m_p * g; mc.c[9] = 2.0 * m_p * l; mc.c[10] = 4.0 * g;
    mc.c[11] = hh * (1.0 / l); mc.c[12] = -(hh * (1.0 / l)); mc.c[13] = 3.0 * m_p * l;
    mc.c[14] = m_c + m_p;
  }
  static void host_consts(const double* p, double hh, ModelConst& mc) {
    mc.hh = hh;
    mc.mhh = -hh;
    mc.one = 1.0;
    mc.mz = -0.0;
    param_consts(p, hh, mc);
  }
  __device__ __forceinline__ static void device_param(ModelConst&, double) {}
  // Parameters from device memory: the constants recomputed (hh, one and mz stay as launched).
  __device__ __forceinline__ static void device_params(ModelConst& K, const double* p) {
    const double q[4] = {__ldg(p), __ldg(p + 1), __ldg(p + 2), __ldg(p + 3)};
    param_consts(q, K.hh, K);
  }

  // With WP (the parameter derivative of J^T w) eval also fills mdp = -hh df/dp, p = (mc, mp, l,
  // g), from the same intermediates (FUSED_DP: the kernels call no separate dparams):
  //   dpdd/dmc = -pdd / D,            dpdd/dmp = s (l w^2 + g c - pdd s) / D,
  //   dpdd/dl  = mp s w^2 / D,        dpdd/dg  = mp s c / D,
  //   dthdd/dmc = -(g s + Bu) / (l D), dthdd/dmp = -s (l w^2 c + g + Bu s) / (l D),
  //   dthdd/dl  = -(mp s w^2 c / D + Bu / l) / l,   dthdd/dg = -(mc + mp) s / (l D)
  // (D_mc = 1, D_mp = s^2; A and B are linear in each parameter).
  static constexpr bool FUSED_DP = true;
  template <bool WC, bool WJ, bool WH, bool WP = false>
  __device__ __forceinline__ static void eval(const ModelConst& K, const double (&z)[NZ], const double (&yb)[NX],
                                              const double (&cqd)[NZ], double (&pa)[NX], double (&pb)[NX],
                                              double (&mjx)[NX][MAXRX], double (&mju)[NX][MAXRU],
                                              double (&hd)[NHD], double (*mdp)[NP] = nullptr) {
    const double mcm = K.c[0], mp = K.c[1], l = K.c[2], g = K.c[3], Mg = K.c[4];
    const double mpl = K.c[6], mp2 = K.c[7], mpg = K.c[8], mpl2 = K.c[9], g4 = K.c[10];
    const double hh = K.hh, mhh = K.mhh;
    const double p = z[0], pd = z[1], th = z[2], w = z[3], F = z[4];
    double s, c;
    sincos_tab(K, th, s, c);
    const double ms = fmul(K, mp, s);
    const double D = fma(ms, s, mcm);
    const double iD = recip(K.one, D);
    const double w2 = fmul(K, w, w);
    const double lw2 = fmul(K, l, w2);
    const double gl = fma(g, c, lw2);             // l w^2 + g c
    const double A = fma(ms, gl, F);
    const double pdd = fmul(K, A, iD);
    const double mplw2 = fmul(K, mpl, w2);
    const double B = fma(-s, fma(mplw2, c, Mg), fmul(K, -F, c));
    const double Bu = fmul(K, B, iD);             // l thdd
    const double hhil = K.c[11], mhhil = K.c[12];
    if (WC) {
      pa[0] = fma(hh, pd, p);   pb[0] = fma(mhh, pd, p);
      pa[1] = fma(hh, pdd, pd); pb[1] = fma(mhh, pdd, pd);
      pa[2] = fma(hh, w, th);   pb[2] = fma(mhh, w, th);
      pa[3] = fma(hhil, Bu, w); pb[3] = fma(mhhil, Bu, w);
    }
    if (WJ || WH) {
      const double sc = fmul(K, s, c);
      const double c2s2 = fma(c, c, fmul(K, -s, s));
      const double Dp = fmul(K, mp2, sc);
      const double A_t = fma(mplw2, c, fmul(K, mpg, c2s2));
      const double pdd_t = fmul(K, fma(-pdd, Dp, A_t), iD);
      const double lw = fmul(K, mpl2, w);          // 2 mp l w
      const double A_w = fmul(K, lw, s);
      const double B_t = fma(F, s, -fma(mplw2, c2s2, fmul(K, Mg, c)));
      const double Bu_t = fmul(K, fma(-Bu, Dp, B_t), iD);
      const double B_w = fmul(K, -lw, sc);
      const double Bu_w = fmul(K, B_w, iD);
      const double Bu_F = fmul(K, -c, iD);
      const double mhiD = fmul(K, mhh, iD);
      if (WJ) {
        mjx[0][0] = 0.0; mjx[0][1] = mhh; mjx[0][2] = 0.0;
        mjx[1][0] = 0.0; mjx[1][1] = fmul(K, mhh, pdd_t); mjx[1][2] = fmul(K, mhiD, A_w);
        mju[1][0] = mhiD;
        mjx[2][0] = 0.0; mjx[2][1] = mhh; mjx[2][2] = 0.0;
        mjx[3][0] = fmul(K, mhhil, Bu_t); mjx[3][1] = fmul(K, mhhil, Bu_w);
        mju[3][0] = fmul(K, mhhil, Bu_F);
      }
      if (WP) {
#pragma unroll
        for (int k = 0; k < NX; ++k)
#pragma unroll
          for (int i = 0; i < NP; ++i) mdp[k][i] = 0.0;
        const double mhhilD = fmul(K, mhhil, iD);
        mdp[1][0] = fmul(K, -mhiD, pdd);
        mdp[1][1] = fmul(K, mhiD, fmul(K, s, fma(-pdd, s, gl)));
        mdp[1][2] = fmul(K, mhiD, fmul(K, ms, w2));
        mdp[1][3] = fmul(K, mhiD, fmul(K, ms, c));
        mdp[3][0] = fmul(K, mhhilD, -fma(g, s, Bu));
        mdp[3][1] = fmul(K, mhhilD, fmul(K, -s, fma(lw2, c, fma(Bu, s, g))));
        mdp[3][2] = fmul(K, mhhil, -fma(fmul(K, ms, fmul(K, w2, c)), iD, fmul(K, Bu, K.c[5])));
        mdp[3][3] = fmul(K, mhhilD, fmul(K, -K.c[14], s));
      }
      if (WH) {
        // Every second derivative above is (numerator) / D: the multipliers carry the 1/D (and
        // for the angular rows the 1/l), m1 = -hh ybar_1 / D and m3 = -hh ybar_3 / (l D), and the
        // numerators are combined directly (those of the angular rows scaled by l).
        const double m1 = fmul(K, mhiD, yb[1]), m3 = fmul(K, fmul(K, mhhil, yb[3]), iD);
        const double Dpp = fmul(K, mp2, c2s2);
        const double mDp2 = fmul(K, -2.0, Dp);
        // A_tt = -mp s (l w^2 + 4 g c)
        const double A_tt = fmul(K, -ms, fma(g4, c, lw2));
        const double n_pdd_tt = fma(-pdd, Dpp, fma(pdd_t, mDp2, A_tt));
        // B_tt = F c + 4 mp l w^2 s c + (mc+mp) g s = -B + 3 mp l w^2 s c
        const double B_tt = fma(sc, fmul(K, K.c[13], w2), -B);
        const double n_bu_tt = fma(-Bu, Dpp, fma(Bu_t, mDp2, B_tt));
        hd[0] = fma(m1, n_pdd_tt, fma(m3, n_bu_tt, cqd[2]));   // (th, th)
        // The other three entries, with t = m3 c - m1 and e = D' / D, from
        //   pdd_ww = 2 mp l s / D,  Bu_ww = -2 mp l s c / D                  -> (w, w)  = -t 2 mp l s
        //   pdd_tF = -e / D,        Bu_tF = (s + c e) / D                     -> (F, th) = m3 s + e t
        //   pdd_tw = 2 mp l w (c - s e) / D,  Bu_tw = -2 mp l w (c^2 - s^2 - s c e) / D
        //                                    -> (w, th) = 2 mp l w (m1 c - m3 (c^2 - s^2) + e s t)
        const double t = fma(m3, c, -m1);
        const double e = fmul(K, Dp, iD);
        hd[1] = fmul(K, lw, fma(fmul(K, e, s), t, fma(m1, c, -fmul(K, m3, c2s2))));   // (w, th)
        hd[2] = fma(-t, fmul(K, mpl2, s), cqd[3]);                                  // (w, w)
        hd[3] = fma(e, t, fmul(K, m3, s));                                          // (F, th)
      }
    }
  }
  __device__ __forceinline__ static void dparam(const ModelConst&, const double (&)[NZ], double (&mdp)[NX]) {
    mdp[0] = mdp[1] = mdp[2] = mdp[3] = 0.0;
  }
  __device__ __forceinline__ static void dparam_grad(const ModelConst&, const double (&)[NZ], const double (&)[NX],
                                                     double (&out)[NZ]) {
    for (int v = 0; v < NZ; ++v) out[v] = 0.0;
  }
};

}  // namespace ocpg
