// Device models of the dynamics x' = f(x, u) (paper Sec. 3) with hand-derived derivatives.
//
// Every model describes, at compile time, the sparsity template of one node:
//   - for each state component k, the Jacobian row template of the defect c_{k,j}: the
//     X-local variables XV(k, .) (sorted, always including k itself for the identity term of
//     the trapezoidal defect) and the U-local variables UV(k, .) whose derivative
//     df_k/dz_v is not identically zero; JZ(k, e) marks entries that are the identity term
//     alone (df_k/dz_v identically 0);
//   - the pairs (HA(e) >= HB(e)) of local variables with a Hessian of some f_k not
//     identically zero, and HK(k): whether f_k has a Hessian at all.
// The host pattern compiler reads these tables; the kernels place values by them.
//
// At one node z = (x, u) a model returns, with hh = h/2:
//   pa[k] = x_k + hh f_k(z),  pb[k] = x_k - hh f_k(z)   (defect (k,j) = pb(j+1) - pa(j))
//   mjx[k][e] = -hh df_k/dx_{XV(k,e)}(z)   (identity excluded),  mju[k][e] = -hh df_k/du_{UV(k,e)}(z)
//   hd[e] = -hh sum_k ybar_k d2 f_k/dz_{HA(e)} dz_{HB(e)}(z)  (+ cqd[a] on a diagonal entry),
// where cqd is the diagonal of sigma * w_j * Hess f0 at this node.  A Jacobian value is then
// mjx - 1 (left node, identity), mjx + 1 (right node, identity) or the bare mjx / mju.
//
// The library is compiled with automatic FMA contraction off: every FMA below is explicit,
// so the FP64 operation count is what the source says (GB300 executes FP64 at 2 FMA per
// clock per SM, which bounds these kernels) and every kernel variant rounds identically.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ocpg {

// Kernel-side model constants (filled by the host from the handle's parameters).
struct ModelConst {
  double hh;       // h / 2
  double mhh;      // -h / 2
  double one;      // 1.0 and -0.0, passed at run time (see fadd / fmul below)
  double mz;
  double c[16];    // model-specific precomputed constants (see each model)
};

// GB300's FP64 pipe sustains FMAs at its full rate but separate adds and multiplies about 18%
// slower (measured), so sums, differences and products are issued as FMAs against the run-time
// constants 1 and -0: a + b = fma(a, 1, b), a - b = fma(-b, 1, a), a * b = fma(a, b, -0).
// These round exactly like the plain operations (signed zeros included); the constants come
// from kernel parameters so that the compiler cannot fold the FMAs back.
__device__ __forceinline__ double fadd(const ModelConst& K, double a, double b) { return fma(a, K.one, b); }
__device__ __forceinline__ double fsub(const ModelConst& K, double a, double b) { return fma(-b, K.one, a); }
__device__ __forceinline__ double fmul(const ModelConst& K, double a, double b) { return fma(a, b, K.mz); }

#define OCP_TABLE1(NAME, TYPE, N, ...)                       \
  __host__ __device__ static constexpr TYPE NAME(int k) {    \
    constexpr TYPE t[N] = __VA_ARGS__;                       \
    return t[k];                                             \
  }
#define OCP_TABLE2(NAME, TYPE, N, M, ...)                        \
  __host__ __device__ static constexpr TYPE NAME(int k, int e) { \
    constexpr TYPE t[N][M] = __VA_ARGS__;                        \
    return t[k][e];                                              \
  }

// ------------------------------------------------------------------------------------
// Van der Pol:  f0 = x2,  f1 = mu (1 - x1^2) x2 - x1 + u.
//   df1/dx1 = -2 mu x1 x2 - 1,  df1/dx2 = mu (1 - x1^2),  df1/du = 1
//   d2f1/dx1^2 = -2 mu x2,  d2f1/dx1dx2 = -2 mu x1
//   df1/dmu = (1 - x1^2) x2,  d2f1/dmu dx1 = -2 x1 x2,  d2f1/dmu dx2 = 1 - x1^2
// Constants: c[0] = 2 hh mu, c[1] = hh mu, c[2] = -hh mu.
// ------------------------------------------------------------------------------------
struct VdP {
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

// ------------------------------------------------------------------------------------
// Double integrator (paper Sec. 5):  f0 = x2,  f1 = u.  Linear: no Hessian.
// ------------------------------------------------------------------------------------
struct Dint {
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

  static void host_consts(const double*, double hh, ModelConst& mc) {
    mc.hh = hh;
    mc.mhh = -hh;
    mc.one = 1.0;
    mc.mz = -0.0;
  }
  __device__ __forceinline__ static void device_param(ModelConst&, double) {}

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
  __device__ __forceinline__ static void dparam_grad(const ModelConst&, const double (&)[NZ], const double (&)[NX],
                                                     double (&out)[NZ]) {
    out[0] = out[1] = out[2] = 0.0;
  }
};

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
//            c[8]=mp g, c[9]=2 mp l, c[10]=4 g.
// ------------------------------------------------------------------------------------
struct CartPole {
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

  static void host_consts(const double* p, double hh, ModelConst& mc) {
    mc.hh = hh;
    mc.mhh = -hh;
    mc.one = 1.0;
    mc.mz = -0.0;
    const double m_c = p[0], m_p = p[1], l = p[2], g = p[3];
    mc.c[0] = m_c; mc.c[1] = m_p; mc.c[2] = l; mc.c[3] = g;
    mc.c[4] = (m_c + m_p) * g; mc.c[5] = 1.0 / l; mc.c[6] = m_p * l; mc.c[7] = 2.0 * m_p;
    mc.c[8] = m_p * g; mc.c[9] = 2.0 * m_p * l; mc.c[10] = 4.0 * g;
  }
  __device__ __forceinline__ static void device_param(ModelConst&, double) {}

  template <bool WC, bool WJ, bool WH>
  __device__ __forceinline__ static void eval(const ModelConst& K, const double (&z)[NZ], const double (&yb)[NX],
                                              const double (&cqd)[NZ], double (&pa)[NX], double (&pb)[NX],
                                              double (&mjx)[NX][MAXRX], double (&mju)[NX][MAXRU],
                                              double (&hd)[NHD]) {
    const double mcm = K.c[0], mp = K.c[1], l = K.c[2], g = K.c[3], Mg = K.c[4], il = K.c[5];
    const double mpl = K.c[6], mp2 = K.c[7], mpg = K.c[8], mpl2 = K.c[9], g4 = K.c[10];
    const double hh = K.hh, mhh = K.mhh;
    const double p = z[0], pd = z[1], th = z[2], w = z[3], F = z[4];
    double s, c;
    sincos(th, &s, &c);
    const double ms = fmul(K, mp, s);
    const double D = fma(ms, s, mcm);
    const double iD = 1.0 / D;
    const double iDl = fmul(K, iD, il);
    const double w2 = fmul(K, w, w);
    const double lw2 = fmul(K, l, w2);
    const double A = fma(ms, fma(g, c, lw2), F);
    const double pdd = fmul(K, A, iD);
    const double mplw2 = fmul(K, mpl, w2);
    const double B = fma(-s, fma(mplw2, c, Mg), fmul(K, -F, c));
    const double thdd = fmul(K, B, iDl);
    if (WC) {
      pa[0] = fma(hh, pd, p);   pb[0] = fma(mhh, pd, p);
      pa[1] = fma(hh, pdd, pd); pb[1] = fma(mhh, pdd, pd);
      pa[2] = fma(hh, w, th);   pb[2] = fma(mhh, w, th);
      pa[3] = fma(hh, thdd, w); pb[3] = fma(mhh, thdd, w);
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
      const double thdd_t = fmul(K, fma(B_t, il, fmul(K, -thdd, Dp)), iD);
      const double B_w = fmul(K, -lw, sc);
      const double thdd_w = fmul(K, B_w, iDl);
      const double thdd_F = fmul(K, -c, iDl);
      if (WJ) {
        const double mhiD = fmul(K, mhh, iD);
        mjx[0][0] = 0.0; mjx[0][1] = mhh; mjx[0][2] = 0.0;
        mjx[1][0] = 0.0; mjx[1][1] = fmul(K, mhh, pdd_t); mjx[1][2] = fmul(K, mhiD, A_w);
        mju[1][0] = mhiD;
        mjx[2][0] = 0.0; mjx[2][1] = mhh; mjx[2][2] = 0.0;
        mjx[3][0] = fmul(K, mhh, thdd_t); mjx[3][1] = fmul(K, mhh, thdd_w);
        mju[3][0] = fmul(K, mhh, thdd_F);
      }
      if (WH) {
        const double pdd_w = fmul(K, A_w, iD);
        const double Dpp = fmul(K, mp2, c2s2);
        const double my1 = fmul(K, mhh, yb[1]), my3 = fmul(K, mhh, yb[3]);
        // A_tt = -mp s (l w^2 + 4 g c)
        const double A_tt = fmul(K, -ms, fma(g4, c, lw2));
        const double pdd_tt = fmul(K, fma(-pdd, Dpp, fma(fmul(K, -2.0, pdd_t), Dp, A_tt)), iD);
        const double A_tw = fmul(K, lw, c);
        const double pdd_tw = fmul(K, fma(-pdd_w, Dp, A_tw), iD);
        const double pdd_ww = fmul(K, fmul(K, mpl2, s), iD);
        const double pdd_tF = fmul(K, fmul(K, -Dp, iD), iD);
        // B_tt = F c + 4 mp l w^2 s c + (mc+mp) g s
        const double B_tt = fma(F, c, fmul(K, s, fma(fmul(K, 4.0, mplw2), c, Mg)));
        const double thdd_tt = fmul(K, fma(-thdd, Dpp, fma(fmul(K, -2.0, thdd_t), Dp, fmul(K, B_tt, il))), iD);
        const double B_tw = fmul(K, -lw, c2s2);
        const double thdd_tw = fmul(K, fma(-thdd_w, Dp, fmul(K, B_tw, il)), iD);
        const double thdd_ww = fmul(K, fmul(K, -mp2, sc), iD);
        const double thdd_tF = fmul(K, fma(-thdd_F, Dp, fmul(K, s, il)), iD);
        hd[0] = fma(my1, pdd_tt, fma(my3, thdd_tt, cqd[2]));   // (th, th)
        hd[1] = fma(my1, pdd_tw, fmul(K, my3, thdd_tw));       // (w, th)
        hd[2] = fma(my1, pdd_ww, fma(my3, thdd_ww, cqd[3]));   // (w, w)
        hd[3] = fma(my1, pdd_tF, fmul(K, my3, thdd_tF));       // (F, th)
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
