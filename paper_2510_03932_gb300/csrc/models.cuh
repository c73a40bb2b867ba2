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
        // Every second derivative above is (numerator) / D: the multipliers carry the 1/D,
        // m1 = -hh ybar_1 / D and m3 = -hh ybar_3 / D, and the numerators are combined directly.
        const double m1 = fmul(K, fmul(K, mhh, yb[1]), iD), m3 = fmul(K, fmul(K, mhh, yb[3]), iD);
        const double pdd_w = fmul(K, A_w, iD);
        const double Dpp = fmul(K, mp2, c2s2);
        const double mDp2 = fmul(K, -2.0, Dp);
        // A_tt = -mp s (l w^2 + 4 g c)
        const double A_tt = fmul(K, -ms, fma(g4, c, lw2));
        const double n_pdd_tt = fma(-pdd, Dpp, fma(pdd_t, mDp2, A_tt));
        const double A_tw = fmul(K, lw, c);
        const double n_pdd_tw = fma(-pdd_w, Dp, A_tw);
        const double n_pdd_ww = fmul(K, mpl2, s);
        const double n_pdd_tF = fmul(K, -Dp, iD);
        // B_tt = F c + 4 mp l w^2 s c + (mc+mp) g s
        const double B_tt = fma(F, c, fmul(K, s, fma(fmul(K, 4.0, mplw2), c, Mg)));
        const double n_thdd_tt = fma(-thdd, Dpp, fma(thdd_t, mDp2, fmul(K, B_tt, il)));
        const double B_tw = fmul(K, -lw, c2s2);
        const double n_thdd_tw = fma(-thdd_w, Dp, fmul(K, B_tw, il));
        const double n_thdd_ww = fmul(K, -mp2, sc);
        const double n_thdd_tF = fma(-thdd_F, Dp, fmul(K, s, il));
        hd[0] = fma(m1, n_pdd_tt, fma(m3, n_thdd_tt, cqd[2]));   // (th, th)
        hd[1] = fma(m1, n_pdd_tw, fmul(K, m3, n_thdd_tw));       // (w, th)
        hd[2] = fma(m1, n_pdd_ww, fma(m3, n_thdd_ww, cqd[3]));   // (w, w)
        hd[3] = fma(m1, n_pdd_tF, fmul(K, m3, n_thdd_tF));       // (F, th)
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

// ------------------------------------------------------------------------------------
// Goddard rocket (the paper's first benchmark problem, appendix): z = (r, v, m, u) =
// (altitude, speed, mass, normalised thrust), params (Cd, beta, Tmax, b):
//   r' = v,  v' = -D - 1/r^2 + u Tmax / m,  m' = -b Tmax u,  D = Cd v^2 exp(-beta (r - 1)) / m.
// Only the sparsity tables live here (for the pattern compiler); the values are computed by
// the dedicated free-final-time kernels (goddard_kernels.cu).
// ------------------------------------------------------------------------------------
struct Goddard {
  static constexpr int EVAL_MIN_CTAS = 0;
  static constexpr int NX = 3, NU = 1, NZ = 4;
  static constexpr int MAXRX = 3, MAXRU = 1;
  OCP_TABLE1(RX, int, NX, {2, 3, 1})
  OCP_TABLE1(RU, int, NX, {0, 1, 1})
  OCP_TABLE2(XV, int, NX, MAXRX, {{0, 1, -1}, {0, 1, 2}, {2, -1, -1}})
  OCP_TABLE2(UV, int, NX, MAXRU, {{-1}, {0}, {0}})
  OCP_TABLE2(JZ, bool, NX, MAXRX, {{true, false, false}, {false, false, false}, {true, false, false}})
  OCP_TABLE1(HK, bool, NX, {false, true, false})
  static constexpr int NHD = 7;
  OCP_TABLE1(HA, int, NHD, {0, 1, 1, 2, 2, 2, 3})
  OCP_TABLE1(HB, int, NHD, {0, 0, 1, 0, 1, 2, 2})
};

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
  static constexpr int EVAL_MIN_CTAS = 6; // 168 registers: measured 14% faster evaluation, 4% faster fused step
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

  static void host_consts(const double* p, double hh, ModelConst& mc) {
    mc.hh = hh;
    mc.mhh = -hh;
    mc.one = 1.0;
    mc.mz = -0.0;
    mc.c[0] = p[0];
  }
  __device__ __forceinline__ static void device_param(ModelConst&, double) {}

  template <bool WC, bool WJ, bool WH>
  __device__ __forceinline__ static void eval(const ModelConst& K, const double (&z)[NZ], const double (&yb)[NX],
                                              const double (&cqd)[NZ], double (&pa)[NX], double (&pb)[NX],
                                              double (&mjx)[NX][MAXRX], double (&mju)[NX][MAXRU],
                                              double (&hd)[NHD]) {
    const double hh = K.hh, mhh = K.mhh;
    const double u1 = z[9], u2 = z[10], u3 = z[11];
    double s7, c7, s8, c8, s9, c9;
    sincos(z[6], &s7, &c7);
    sincos(z[7], &s8, &c8);
    sincos(z[8], &s9, &c9);
    const double e = 1.0 / c8;
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
  __device__ __forceinline__ static void dparam_grad(const ModelConst&, const double (&)[NZ], const double (&)[NX],
                                                     double (&out)[NZ]) {
    for (int v = 0; v < NZ; ++v) out[v] = 0.0;
  }
};

}  // namespace ocpg
