/*
 * CPU ORACLE for the trapezoidal direct transcription of an optimal control problem.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously-correct FP64 statement of
 * what the CUDA library computes.  Only the test-suite, the package smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header, table or
 * helper with the CUDA library, and neither side includes or links the other.
 *
 * What it computes (paper sections in brackets):
 *   - the NLP unknown vector  x = [X_0..X_N (nx each, node-major); U_0..U_N (nu each)]
 *     (Sec. 3 unknown vector; Sec. 5: the state is an nx x (N+1) array, controls after it;
 *      the trapezoid cost uses u at j = 0..N, so controls live on N+1 nodes);
 *   - constraints, in declaration order: the initial boundary rows x(0) (the expression
 *     X_{0,k}, bounds lcon = ucon = x0, Sec. 5), optional final rows X_{N,k}, then one
 *     block of N trapezoidal defects per state component (Sec. 5 defect generator):
 *         c_{k,j} = (X_{j+1,k} - X_{j,k}) - h (f_k(z_j) + f_k(z_{j+1})) / 2 ,  row nb + k N + j;
 *   - objective: the trapezoidal Lagrange cost (Sec. 5, two objective generators summed),
 *         F = sum_j w_j f0(z_j),  w_0 = w_N = h/2,  w_j = h otherwise,  h = T/N (uniform grid);
 *   - gradient of F, the Jacobian of c, and the Lagrangian Hessian
 *         H = sigma * Hess F + sum_r y_r Hess c_r   (lower triangle)
 *     as COO with one entry per structural nonzero, sorted by (row, col);
 *   - the products J v, J^T w, H v, defined as plain COO matrix-vector products;
 *   - (dc/dp)^T w for every dynamics parameter p (Van der Pol mu; cart-pole mc, mp, l, g;
 *     Goddard Cd, beta, Tmax, b; quadrotor g): only the defect rows depend on p.
 *
 * Models: Van der Pol, cart-pole, the heat equation by the method of lines, the Sec. 5
 * double integrator and the Goddard rocket and quadrotor of the paper's appendix.  The running cost is a
 * diagonal quadratic around a reference; the state reference may vary in time as
 * xref_k + xslope_k t + xamp_k sin(xfreq_k t) (the quadrotor's tracking terms), evaluated at
 * the node times t_j = j h.
 *
 * Derivatives of the model right-hand sides are derived by hand and written out in
 * straight-line code (quotient rule for the cart-pole).  Everything is templated on the
 * scalar type so that the same code runs in
 *   - double                 (the oracle values),
 *   - std::complex<double>   (complex-step derivatives used by the tests to pin the
 *                             hand-derived derivatives against the residual itself),
 *   - Sh                     (a running error bound: value v plus magnitude m such that the
 *                             rounding error of v is about u*m; used for the tolerance gate
 *                             of entries that suffer cancellation).
 * The objective and the (dc/dp)^T w reduction use Neumaier compensated summation.
 * Build: g++ -O2 -ffp-contract=off (no FMA contraction, host libm for sin/cos).
 */
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <map>
#include <utility>
#include <vector>

namespace orc {

// ---------------------------------------------------------------------------------------
// Scalar types
// ---------------------------------------------------------------------------------------
struct Sh {  // running error analysis: |computed - exact| <~ u * m
  double v, m;
  Sh(double value = 0.0, double mag = 0.0) : v(value), m(mag) {}
};
inline Sh operator+(Sh a, Sh b) { double v = a.v + b.v; return Sh(v, a.m + b.m + std::fabs(v)); }
inline Sh operator-(Sh a, Sh b) { double v = a.v - b.v; return Sh(v, a.m + b.m + std::fabs(v)); }
inline Sh operator-(Sh a) { return Sh(-a.v, a.m); }
inline Sh operator*(Sh a, Sh b) {
  double v = a.v * b.v;
  return Sh(v, std::fabs(b.v) * a.m + std::fabs(a.v) * b.m + std::fabs(v));
}
inline Sh operator/(Sh a, Sh b) {
  double v = a.v / b.v;
  return Sh(v, (a.m + std::fabs(v) * b.m) / std::fabs(b.v) + std::fabs(v));
}
inline Sh& operator+=(Sh& a, Sh b) { a = a + b; return a; }
inline Sh sin(Sh a) { return Sh(std::sin(a.v), std::fabs(std::cos(a.v)) * a.m + std::fabs(std::sin(a.v))); }
inline Sh cos(Sh a) { return Sh(std::cos(a.v), std::fabs(std::sin(a.v)) * a.m + std::fabs(std::cos(a.v))); }
inline Sh exp(Sh a) {
  const double e = std::exp(a.v);
  return Sh(e, e * a.m + e);
}
inline Sh tan(Sh a) {
  const double t = std::tan(a.v);
  return Sh(t, (1.0 + t * t) * a.m + std::fabs(t));
}

typedef std::complex<double> Cx;

inline double mag(double a) { return std::fabs(a); }
inline double mag(const Cx& a) { return std::fabs(a.real()); }
inline double mag(const Sh& a) { return std::fabs(a.v); }

inline double val(double a) { return a; }
inline double val(const Sh& a) { return a.v; }
inline double shadow(const Sh& a) { return a.m; }

// Neumaier (1974) compensated summation.
template <class S>
struct Neumaier {
  S sum = S(0.0), comp = S(0.0);
  void add(const S& t) {
    S s = sum + t;
    if (mag(sum) >= mag(t)) comp += (sum - s) + t;
    else comp += (t - s) + sum;
    sum = s;
  }
  S result() const { return sum + comp; }
};

// ---------------------------------------------------------------------------------------
// Problem description (mirrored by a ctypes Structure in oracle.py)
// ---------------------------------------------------------------------------------------
enum { M_VDP = 1, M_CARTPOLE = 2, M_HEAT = 3, M_DINT = 4, M_QUAD = 5, M_GODDARD = 6 };

struct Prob {
  int32_t model, nx, nu, has_final;
  int64_t N;
  double T;
  double par[8];
  int32_t npar, pad;
  const double* q;     // running cost weights on the state (nx)
  const double* r;     // running cost weights on the control (nu)
  const double* xref;  // state reference (nx)
  const double* uref;  // control reference (nu)
  // time-varying state reference (each nullable, nx):
  //   xref_k(t) = xref_k + xslope_k t + xamp_k sin(xfreq_k t)
  const double* xslope;
  const double* xamp;
  const double* xfreq;
  // free final time: the horizon tf is an unknown appended to x (h = tf / N); T is unused
  int32_t free_tf;
  // final rows X_{N,k} for the nfin components fin_comp[] (ascending); when has_final is set
  // and fin_comp is null, every component has a final row
  int32_t nfin;
  const int32_t* fin_comp;
  // linear terminal (Mayer) cost sum_k mayer_k X_{N,k} added to the objective (nullable, nx)
  const double* mayer;
  // one-step scheme: 0 trapezoidal (controls on N+1 nodes), 1 forward Euler (paper Sec. 3:
  // controls U_0..U_{N-1}, rectangle-rule cost)
  int32_t scheme;
  // path inequalities (paper Sec. 3) c_p(z_i) <= 0 at every node with a control, p < npath:
  //   c_p(z) = sum_v [ path_a[p,v] (z_v - path_b[p,v])^2 + path_l[p,v] z_v ] - path_r[p]
  // (arrays npath x (nx+nu) row-major, and npath)
  int32_t npath;
  const double* path_a;
  const double* path_b;
  const double* path_l;
  const double* path_r;
  // boundary inequalities (paper Sec. 3) b_q(X_0, X_N) <= 0, q < nbin, on z = (X_0, X_N):
  //   b_q(z) = sum_v [ bin_a[q,v] (z_v - bin_b[q,v])^2 + bin_l[q,v] z_v ] - bin_r[q]
  // (arrays nbin x 2 nx row-major: columns 0..nx-1 are X_0, nx..2nx-1 are X_N; and nbin)
  int32_t nbin;
  const double* bin_a;
  const double* bin_b;
  const double* bin_l;
  const double* bin_r;
  // boundary cost (paper Sec. 3, the Bolza term g(X_0, X_N)) added to the objective:
  //   g(z) = sum_v [ bol_a[v] (z_v - bol_b[v])^2 + bol_l[v] z_v ],  z = (X_0, X_N)
  // (arrays of 2 nx; has_bol = 0: none)
  int32_t has_bol;
  const double* bol_a;
  const double* bol_b;
  const double* bol_l;
};

template <class S> struct JEnt { int k, v; S val; };      // d f_k / d z_v
template <class S> struct HEnt { int k, a, b; S val; };   // d2 f_k / d z_a d z_b, a >= b

// ---------------------------------------------------------------------------------------
// Models.  z = (x_1..x_nx, u_1..u_nu) at one node; p = parameters.
// Every structural entry is emitted whatever its value at z.
// ---------------------------------------------------------------------------------------

// Van der Pol: x1' = x2, x2' = mu (1 - x1^2) x2 - x1 + u ; p = (mu).
template <class S> void vdp_f(const S* p, const S* z, S* f) {
  const S mu = p[0], x1 = z[0], x2 = z[1], u = z[2];
  f[0] = x2;
  f[1] = mu * (S(1.0) - x1 * x1) * x2 - x1 + u;
}
template <class S> void vdp_jac(const S* p, const S* z, std::vector<JEnt<S>>& e) {
  const S mu = p[0], x1 = z[0], x2 = z[1];
  e.push_back({0, 1, S(1.0)});
  e.push_back({1, 0, S(-2.0) * mu * x1 * x2 - S(1.0)});
  e.push_back({1, 1, mu * (S(1.0) - x1 * x1)});
  e.push_back({1, 2, S(1.0)});
}
template <class S> void vdp_hess(const S* p, const S* z, std::vector<HEnt<S>>& e) {
  const S mu = p[0], x1 = z[0], x2 = z[1];
  e.push_back({1, 0, 0, S(-2.0) * mu * x2});
  e.push_back({1, 1, 0, S(-2.0) * mu * x1});
}
template <class S> void vdp_dpar(const S* p, const S* z, S* d) {
  (void)p;
  const S x1 = z[0], x2 = z[1];
  d[0] = S(0.0);
  d[1] = (S(1.0) - x1 * x1) * x2;
}

// Cart-pole with a point-mass pole of length l, theta measured from the downward vertical.
// Euler-Lagrange equations of L = 1/2 (mc+mp) pd^2 + mp l pd w cos(th) + 1/2 mp l^2 w^2
// + mp g l cos(th), with the force F on the cart, solved for the accelerations:
//   D  = mc + mp sin^2(th)
//   p'' = (F + mp sin(th) (l w^2 + g cos(th))) / D
//   th''= (-F cos(th) - mp l w^2 cos(th) sin(th) - (mc+mp) g sin(th)) / (l D)
// state z = (p, pd, th, w, F);  p = (mc, mp, l, g).
template <class S> void cp_f(const S* p, const S* z, S* f) {
  using std::cos; using std::sin;
  const S mc = p[0], mp = p[1], l = p[2], g = p[3];
  const S pd = z[1], th = z[2], w = z[3], F = z[4];
  const S s = sin(th), c = cos(th);
  const S D = mc + mp * s * s;
  f[0] = pd;
  f[1] = (F + mp * s * (l * w * w + g * c)) / D;
  f[2] = w;
  f[3] = (S(0.0) - F * c - mp * l * w * w * c * s - (mc + mp) * g * s) / (l * D);
}

// Quotient rule for q = A / D with D depending on th only (local variables th, w, F):
//   q_a  = A_a / D - A D_a / D^2
//   q_ab = A_ab / D - (A_a D_b + A_b D_a) / D^2 - A D_ab / D^2 + 2 A D_a D_b / D^3
template <class S> void cp_parts(const S* p, const S* z,
                                 S& A, S& A_t, S& A_w, S& A_F, S& A_tt, S& A_tw, S& A_ww, S& A_tF,
                                 S& B, S& B_t, S& B_w, S& B_F, S& B_tt, S& B_tw, S& B_ww, S& B_tF,
                                 S& D, S& D_t, S& D_tt, S& E, S& E_t, S& E_tt) {
  using std::cos; using std::sin;
  const S mc = p[0], mp = p[1], l = p[2], g = p[3];
  const S th = z[2], w = z[3], F = z[4];
  const S s = sin(th), c = cos(th);
  // numerator of p'':  A = F + mp l w^2 s + mp g s c
  A = F + mp * s * (l * w * w + g * c);
  A_t = mp * l * w * w * c + mp * g * (c * c - s * s);
  A_w = S(2.0) * mp * l * w * s;
  A_F = S(1.0);
  A_tt = S(0.0) - mp * l * w * w * s - S(4.0) * mp * g * s * c;
  A_tw = S(2.0) * mp * l * w * c;
  A_ww = S(2.0) * mp * l * s;
  A_tF = S(0.0);
  // numerator of th'':  B = -F c - mp l w^2 c s - (mc+mp) g s
  B = S(0.0) - F * c - mp * l * w * w * c * s - (mc + mp) * g * s;
  B_t = F * s - mp * l * w * w * (c * c - s * s) - (mc + mp) * g * c;
  B_w = S(-2.0) * mp * l * w * c * s;
  B_F = S(0.0) - c;
  B_tt = F * c + S(4.0) * mp * l * w * w * s * c + (mc + mp) * g * s;
  B_tw = S(-2.0) * mp * l * w * (c * c - s * s);
  B_ww = S(-2.0) * mp * l * c * s;
  B_tF = s;
  // denominators
  D = mc + mp * s * s;
  D_t = S(2.0) * mp * s * c;
  D_tt = S(2.0) * mp * (c * c - s * s);
  E = l * D;
  E_t = l * D_t;
  E_tt = l * D_tt;
}

template <class S> void cp_jac(const S* p, const S* z, std::vector<JEnt<S>>& e) {
  S A, A_t, A_w, A_F, A_tt, A_tw, A_ww, A_tF, B, B_t, B_w, B_F, B_tt, B_tw, B_ww, B_tF, D, D_t, D_tt, E, E_t, E_tt;
  cp_parts(p, z, A, A_t, A_w, A_F, A_tt, A_tw, A_ww, A_tF, B, B_t, B_w, B_F, B_tt, B_tw, B_ww, B_tF,
           D, D_t, D_tt, E, E_t, E_tt);
  e.push_back({0, 1, S(1.0)});
  e.push_back({1, 2, A_t / D - A * D_t / (D * D)});
  e.push_back({1, 3, A_w / D});
  e.push_back({1, 4, A_F / D});
  e.push_back({2, 3, S(1.0)});
  e.push_back({3, 2, B_t / E - B * E_t / (E * E)});
  e.push_back({3, 3, B_w / E});
  e.push_back({3, 4, B_F / E});
}

template <class S> void cp_hess(const S* p, const S* z, std::vector<HEnt<S>>& e) {
  S A, A_t, A_w, A_F, A_tt, A_tw, A_ww, A_tF, B, B_t, B_w, B_F, B_tt, B_tw, B_ww, B_tF, D, D_t, D_tt, E, E_t, E_tt;
  cp_parts(p, z, A, A_t, A_w, A_F, A_tt, A_tw, A_ww, A_tF, B, B_t, B_w, B_F, B_tt, B_tw, B_ww, B_tF,
           D, D_t, D_tt, E, E_t, E_tt);
  // local indices: th = 2, w = 3, F = 4; only D depends on th (D_w = D_F = 0)
  const S D2 = D * D, D3 = D * D * D, E2 = E * E, E3 = E * E * E;
  e.push_back({1, 2, 2, A_tt / D - (A_t * D_t + A_t * D_t) / D2 - A * D_tt / D2 + S(2.0) * A * D_t * D_t / D3});
  e.push_back({1, 3, 2, A_tw / D - A_w * D_t / D2});
  e.push_back({1, 3, 3, A_ww / D});
  e.push_back({1, 4, 2, A_tF / D - A_F * D_t / D2});
  e.push_back({3, 2, 2, B_tt / E - (B_t * E_t + B_t * E_t) / E2 - B * E_tt / E2 + S(2.0) * B * E_t * E_t / E3});
  e.push_back({3, 3, 2, B_tw / E - B_w * E_t / E2});
  e.push_back({3, 3, 3, B_ww / E});
  e.push_back({3, 4, 2, B_tF / E - B_F * E_t / E2});
}

// Heat equation by the method of lines on n cells of width dx = 1/n:
//   x_k' = (x_{k-1} - 2 x_k + x_{k+1}) / dx^2 - x_k^3,
// left ghost x_0 = u (Dirichlet control), right ghost x_{n+1} = x_n (homogeneous Neumann).
// Local indices: cell k (1-based) is z[k-1], the control is z[n].
template <class S> void heat_f(int n, const S* z, S* f) {
  const double dx = 1.0 / n;
  for (int k = 0; k < n; ++k) {
    const S left = (k == 0) ? z[n] : z[k - 1];
    const S right = (k == n - 1) ? z[n - 1] : z[k + 1];
    f[k] = (left - S(2.0) * z[k] + right) / S(dx * dx) - z[k] * z[k] * z[k];
  }
}
template <class S> void heat_jac(int n, const S* z, std::vector<JEnt<S>>& e) {
  const double dx = 1.0 / n;
  const S inv = S(1.0) / S(dx * dx);
  for (int k = 0; k < n; ++k) {
    const int left = (k == 0) ? n : k - 1;
    e.push_back({k, left, inv});
    if (k < n - 1) {
      e.push_back({k, k, S(-2.0) * inv - S(3.0) * z[k] * z[k]});
      e.push_back({k, k + 1, inv});
    } else {
      e.push_back({k, k, S(-1.0) * inv - S(3.0) * z[k] * z[k]});
    }
  }
}
template <class S> void heat_hess(int n, const S* z, std::vector<HEnt<S>>& e) {
  for (int k = 0; k < n; ++k) e.push_back({k, k, k, S(-6.0) * z[k]});
}

// Double integrator: x1' = x2, x2' = u.
template <class S> void dint_f(const S* z, S* f) { f[0] = z[1]; f[1] = z[2]; }
template <class S> void dint_jac(std::vector<JEnt<S>>& e) {
  e.push_back({0, 1, S(1.0)});
  e.push_back({1, 2, S(1.0)});
}

// Goddard rocket (paper appendix, the first benchmark problem): state (r, v, m) = altitude,
// speed and mass, control u = normalised thrust; p = (Cd, beta, Tmax, b):
//   r' = v,
//   v' = -Cd v^2 exp(-beta (r - 1)) / m - 1 / r^2 + u Tmax / m,
//   m' = -b Tmax u.
// With E = exp(-beta (r - 1)) and D = Cd v^2 E / m (the drag term), dD/dr = -beta D,
// dD/dv = 2 Cd v E / m, dD/dm = -D / m; so dv'/dm = D / m - u Tmax / m^2 and
// d2v'/dm2 = 2 (u Tmax / m - D) / m^2.
template <class S> void god_f(const S* p, const S* z, S* f) {
  using std::exp;
  const S Cd = p[0], beta = p[1], Tmax = p[2], b = p[3];
  const S r = z[0], v = z[1], m = z[2], u = z[3];
  f[0] = v;
  f[1] = S(0.0) - Cd * v * v * exp(S(0.0) - beta * (r - S(1.0))) / m - S(1.0) / (r * r) + u * Tmax / m;
  f[2] = S(0.0) - b * Tmax * u;
}
template <class S> void god_jac(const S* p, const S* z, std::vector<JEnt<S>>& e) {
  using std::exp;
  const S Cd = p[0], beta = p[1], Tmax = p[2], b = p[3];
  const S r = z[0], v = z[1], m = z[2], u = z[3];
  const S E = exp(S(0.0) - beta * (r - S(1.0)));
  const S D = Cd * v * v * E / m;
  e.push_back({0, 1, S(1.0)});
  e.push_back({1, 0, beta * D + S(2.0) / (r * r * r)});
  e.push_back({1, 1, S(0.0) - S(2.0) * Cd * v * E / m});
  e.push_back({1, 2, (D - u * Tmax / m) / m});
  e.push_back({1, 3, Tmax / m});
  e.push_back({2, 3, S(0.0) - b * Tmax});
}
template <class S> void god_hess(const S* p, const S* z, std::vector<HEnt<S>>& e) {
  using std::exp;
  const S Cd = p[0], beta = p[1], Tmax = p[2];
  const S r = z[0], v = z[1], m = z[2], u = z[3];
  const S E = exp(S(0.0) - beta * (r - S(1.0)));
  const S D = Cd * v * v * E / m;
  e.push_back({1, 0, 0, S(0.0) - beta * beta * D - S(6.0) / (r * r * r * r)});
  e.push_back({1, 1, 0, S(2.0) * beta * Cd * v * E / m});
  e.push_back({1, 1, 1, S(0.0) - S(2.0) * Cd * E / m});
  e.push_back({1, 2, 0, S(0.0) - beta * D / m});
  e.push_back({1, 2, 1, S(2.0) * Cd * v * E / (m * m)});
  e.push_back({1, 2, 2, S(2.0) * (u * Tmax / m - D) / (m * m)});
  e.push_back({1, 3, 2, S(0.0) - Tmax / (m * m)});
}

// Quadrotor (paper appendix, the second benchmark problem).  States x1..x9: positions
// x1, x3, x5 with velocities x2, x4, x6 and the attitude angles x7, x8, x9; controls u1 (the
// thrust per unit mass) and u2, u3, u4 (angular rate inputs); p = (g).
//   x2' = u1 P,  x4' = u1 Q,  x6' = u1 R - g   with the thrust direction
//     P = cos x7 sin x8 cos x9 + sin x7 sin x9,  Q = cos x7 sin x8 sin x9 - sin x7 cos x9,
//     R = cos x7 cos x8;
//   x7' = (u2 cos x7 + u3 sin x7) / cos x8,  x8' = -u2 sin x7 + u3 cos x7,
//   x9' = (u2 cos x7 + u3 sin x7) tan x8 + u4.
// Local indices: x1..x9 -> 0..8, u1..u4 -> 9..12.
template <class S> void quad_f(const S* p, const S* z, S* f) {
  using std::cos; using std::sin; using std::tan;
  const S g = p[0];
  const S x7 = z[6], x8 = z[7], x9 = z[8], u1 = z[9], u2 = z[10], u3 = z[11], u4 = z[12];
  f[0] = z[1];
  f[1] = u1 * (cos(x7) * sin(x8) * cos(x9) + sin(x7) * sin(x9));
  f[2] = z[3];
  f[3] = u1 * (cos(x7) * sin(x8) * sin(x9) - sin(x7) * cos(x9));
  f[4] = z[5];
  f[5] = u1 * cos(x7) * cos(x8) - g;
  f[6] = (u2 * cos(x7) + u3 * sin(x7)) / cos(x8);
  f[7] = u3 * cos(x7) - u2 * sin(x7);
  f[8] = (u2 * cos(x7) + u3 * sin(x7)) * tan(x8) + u4;
}

// Trigonometric parts shared by the derivatives:  a = u2 c7 + u3 s7 (so x7' = a / c8),
// b = da/dx7 = u3 c7 - u2 s7 (= x8'), e = 1 / c8, t = tan x8 (de/dx8 = e t, dt/dx8 = e^2).
template <class S> struct QuadParts {
  S s7, c7, s8, c8, s9, c9, e, t, a, b, P, P7, P8, P9, Q, Q7, Q8, Q9;
  QuadParts(const S* z) {
    using std::cos; using std::sin; using std::tan;
    s7 = sin(z[6]); c7 = cos(z[6]); s8 = sin(z[7]); c8 = cos(z[7]); s9 = sin(z[8]); c9 = cos(z[8]);
    e = S(1.0) / c8;
    t = tan(z[7]);
    a = z[10] * c7 + z[11] * s7;
    b = z[11] * c7 - z[10] * s7;
    P = c7 * s8 * c9 + s7 * s9;
    P7 = c7 * s9 - s7 * s8 * c9;
    P8 = c7 * c8 * c9;
    P9 = s7 * c9 - c7 * s8 * s9;
    Q = c7 * s8 * s9 - s7 * c9;
    Q7 = S(0.0) - s7 * s8 * s9 - c7 * c9;
    Q8 = c7 * c8 * s9;
    Q9 = c7 * s8 * c9 + s7 * s9;
  }
};

template <class S> void quad_jac(const S* z, std::vector<JEnt<S>>& e) {
  const QuadParts<S> q(z);
  const S u1 = z[9];
  e.push_back({0, 1, S(1.0)});
  e.push_back({1, 6, u1 * q.P7});
  e.push_back({1, 7, u1 * q.P8});
  e.push_back({1, 8, u1 * q.P9});
  e.push_back({1, 9, q.P});
  e.push_back({2, 3, S(1.0)});
  e.push_back({3, 6, u1 * q.Q7});
  e.push_back({3, 7, u1 * q.Q8});
  e.push_back({3, 8, u1 * q.Q9});
  e.push_back({3, 9, q.Q});
  e.push_back({4, 5, S(1.0)});
  e.push_back({5, 6, S(0.0) - u1 * q.s7 * q.c8});
  e.push_back({5, 7, S(0.0) - u1 * q.c7 * q.s8});
  e.push_back({5, 9, q.c7 * q.c8});
  e.push_back({6, 6, q.b * q.e});
  e.push_back({6, 7, q.a * q.e * q.t});
  e.push_back({6, 10, q.c7 * q.e});
  e.push_back({6, 11, q.s7 * q.e});
  e.push_back({7, 6, S(0.0) - q.a});
  e.push_back({7, 10, S(0.0) - q.s7});
  e.push_back({7, 11, q.c7});
  e.push_back({8, 6, q.b * q.t});
  e.push_back({8, 7, q.a * q.e * q.e});
  e.push_back({8, 10, q.c7 * q.t});
  e.push_back({8, 11, q.s7 * q.t});
  e.push_back({8, 12, S(1.0)});
}

template <class S> void quad_hess(const S* z, std::vector<HEnt<S>>& e) {
  const QuadParts<S> q(z);
  const S u1 = z[9];
  // x2' = u1 P:  P_77 = P_99 = -P,  P_78 = -s7 c8 c9,  P_79 = s7 s8 s9 + c7 c9,
  //              P_88 = -c7 s8 c9,  P_89 = -c7 c8 s9
  e.push_back({1, 6, 6, S(0.0) - u1 * q.P});
  e.push_back({1, 7, 6, S(0.0) - u1 * q.s7 * q.c8 * q.c9});
  e.push_back({1, 7, 7, S(0.0) - u1 * q.c7 * q.s8 * q.c9});
  e.push_back({1, 8, 6, u1 * (q.s7 * q.s8 * q.s9 + q.c7 * q.c9)});
  e.push_back({1, 8, 7, S(0.0) - u1 * q.c7 * q.c8 * q.s9});
  e.push_back({1, 8, 8, S(0.0) - u1 * q.P});
  e.push_back({1, 9, 6, q.P7});
  e.push_back({1, 9, 7, q.P8});
  e.push_back({1, 9, 8, q.P9});
  // x4' = u1 Q:  Q_77 = Q_99 = -Q,  Q_78 = -s7 c8 s9,  Q_79 = c7 s9 - s7 s8 c9,
  //              Q_88 = -c7 s8 s9,  Q_89 = c7 c8 c9
  e.push_back({3, 6, 6, S(0.0) - u1 * q.Q});
  e.push_back({3, 7, 6, S(0.0) - u1 * q.s7 * q.c8 * q.s9});
  e.push_back({3, 7, 7, S(0.0) - u1 * q.c7 * q.s8 * q.s9});
  e.push_back({3, 8, 6, u1 * (q.c7 * q.s9 - q.s7 * q.s8 * q.c9)});
  e.push_back({3, 8, 7, u1 * q.c7 * q.c8 * q.c9});
  e.push_back({3, 8, 8, S(0.0) - u1 * q.Q});
  e.push_back({3, 9, 6, q.Q7});
  e.push_back({3, 9, 7, q.Q8});
  e.push_back({3, 9, 8, q.Q9});
  // x6' = u1 c7 c8 - g
  e.push_back({5, 6, 6, S(0.0) - u1 * q.c7 * q.c8});
  e.push_back({5, 7, 6, u1 * q.s7 * q.s8});
  e.push_back({5, 7, 7, S(0.0) - u1 * q.c7 * q.c8});
  e.push_back({5, 9, 6, S(0.0) - q.s7 * q.c8});
  e.push_back({5, 9, 7, S(0.0) - q.c7 * q.s8});
  // x7' = a e
  e.push_back({6, 6, 6, S(0.0) - q.a * q.e});
  e.push_back({6, 7, 6, q.b * q.e * q.t});
  e.push_back({6, 7, 7, q.a * q.e * (q.t * q.t + q.e * q.e)});
  e.push_back({6, 10, 6, S(0.0) - q.s7 * q.e});
  e.push_back({6, 10, 7, q.c7 * q.e * q.t});
  e.push_back({6, 11, 6, q.c7 * q.e});
  e.push_back({6, 11, 7, q.s7 * q.e * q.t});
  // x8' = b
  e.push_back({7, 6, 6, S(0.0) - q.b});
  e.push_back({7, 10, 6, S(0.0) - q.c7});
  e.push_back({7, 11, 6, S(0.0) - q.s7});
  // x9' = a t + u4
  e.push_back({8, 6, 6, S(0.0) - q.a * q.t});
  e.push_back({8, 7, 6, q.b * q.e * q.e});
  e.push_back({8, 7, 7, S(2.0) * q.a * q.e * q.e * q.t});
  e.push_back({8, 10, 6, S(0.0) - q.s7 * q.t});
  e.push_back({8, 10, 7, q.c7 * q.e * q.e});
  e.push_back({8, 11, 6, q.c7 * q.t});
  e.push_back({8, 11, 7, q.s7 * q.e * q.e});
}

// Derivatives of the right-hand sides in the dynamics parameters, d[k * np + i] = df_k / dp_i,
// from the model equations above (np parameters per model: Van der Pol mu; cart-pole mc, mp,
// l, g; Goddard Cd, beta, Tmax, b; quadrotor g).
//
// Cart-pole, with A, B and D as in cp_f and E = l D:  p'' = A / D,  th'' = B / E, and
//   A_mc = 0,  A_mp = s (l w^2 + g c),  A_l = mp s w^2,  A_g = mp s c;  D_mc = 1, D_mp = s^2;
//   B_mc = -g s,  B_mp = -l w^2 c s - g s,  B_l = -mp w^2 c s,  B_g = -(mc + mp) s;
//   E_mc = l,  E_mp = l s^2,  E_l = D,  E_g = 0;
// so dp''/dq = A_q / D - A D_q / D^2 and dth''/dq = B_q / E - B E_q / E^2.
template <class S> void cp_dpar(const S* p, const S* z, S* d) {
  using std::cos; using std::sin;
  const S mc = p[0], mp = p[1], l = p[2], g = p[3];
  const S th = z[2], w = z[3], F = z[4];
  const S s = sin(th), c = cos(th);
  const S D = mc + mp * s * s, E = l * D;
  const S A = F + mp * s * (l * w * w + g * c);
  const S B = S(0.0) - F * c - mp * l * w * w * c * s - (mc + mp) * g * s;
  const S D2 = D * D, E2 = E * E;
  for (int i = 0; i < 16; ++i) d[i] = S(0.0);
  d[4 * 1 + 0] = S(0.0) - A * S(1.0) / D2;
  d[4 * 1 + 1] = s * (l * w * w + g * c) / D - A * (s * s) / D2;
  d[4 * 1 + 2] = mp * s * w * w / D;
  d[4 * 1 + 3] = mp * s * c / D;
  d[4 * 3 + 0] = (S(0.0) - g * s) / E - B * l / E2;
  d[4 * 3 + 1] = (S(0.0) - l * w * w * c * s - g * s) / E - B * (l * s * s) / E2;
  d[4 * 3 + 2] = (S(0.0) - mp * w * w * c * s) / E - B * D / E2;
  d[4 * 3 + 3] = (S(0.0) - (mc + mp) * s) / E;
}
// Goddard:  dv'/dCd = -v^2 exp(-beta (r - 1)) / m,  dv'/dbeta = Cd v^2 (r - 1) exp(-beta (r - 1)) / m,
// dv'/dTmax = u / m;  dm'/dTmax = -b u,  dm'/db = -Tmax u;  r' = v has none.
template <class S> void god_dpar(const S* p, const S* z, S* d) {
  using std::exp;
  const S Cd = p[0], beta = p[1], Tmax = p[2], b = p[3];
  const S r = z[0], v = z[1], m = z[2], u = z[3];
  const S E = exp(S(0.0) - beta * (r - S(1.0)));
  for (int i = 0; i < 12; ++i) d[i] = S(0.0);
  d[4 * 1 + 0] = S(0.0) - v * v * E / m;
  d[4 * 1 + 1] = Cd * v * v * (r - S(1.0)) * E / m;
  d[4 * 1 + 2] = u / m;
  d[4 * 2 + 2] = S(0.0) - b * u;
  d[4 * 2 + 3] = S(0.0) - Tmax * u;
}
// Quadrotor: only x6' = u1 R - g depends on g.
template <class S> void quad_dpar(const S* z, S* d) {
  (void)z;
  for (int k = 0; k < 9; ++k) d[k] = S(0.0);
  d[5] = S(-1.0);
}

// Dispatch ------------------------------------------------------------------------------
template <class S> void model_f(const Prob& P, const S* p, const S* z, S* f) {
  switch (P.model) {
    case M_VDP: vdp_f(p, z, f); break;
    case M_CARTPOLE: cp_f(p, z, f); break;
    case M_HEAT: heat_f(P.nx, z, f); break;
    case M_DINT: dint_f(z, f); break;
    case M_QUAD: quad_f(p, z, f); break;
    case M_GODDARD: god_f(p, z, f); break;
  }
}
template <class S> void model_jac(const Prob& P, const S* p, const S* z, std::vector<JEnt<S>>& e) {
  switch (P.model) {
    case M_VDP: vdp_jac(p, z, e); break;
    case M_CARTPOLE: cp_jac(p, z, e); break;
    case M_HEAT: heat_jac(P.nx, z, e); break;
    case M_DINT: dint_jac(e); break;
    case M_QUAD: quad_jac(z, e); break;
    case M_GODDARD: god_jac(p, z, e); break;
  }
}
template <class S> void model_hess(const Prob& P, const S* p, const S* z, std::vector<HEnt<S>>& e) {
  switch (P.model) {
    case M_VDP: vdp_hess(p, z, e); break;
    case M_CARTPOLE: cp_hess(p, z, e); break;
    case M_HEAT: heat_hess(P.nx, z, e); break;
    case M_DINT: break;
    case M_QUAD: quad_hess(z, e); break;
    case M_GODDARD: god_hess(p, z, e); break;
  }
}

// Number of dynamics parameters with a derivative (the heat cell count is structural; the
// double integrator has none).
inline int model_npar(const Prob& P) {
  switch (P.model) {
    case M_VDP: return 1;
    case M_CARTPOLE: return 4;
    case M_GODDARD: return 4;
    case M_QUAD: return 1;
  }
  return 0;
}
template <class S> void model_dpar(const Prob& P, const S* p, const S* z, S* d) {
  switch (P.model) {
    case M_VDP: vdp_dpar(p, z, d); break;
    case M_CARTPOLE: cp_dpar(p, z, d); break;
    case M_GODDARD: god_dpar(p, z, d); break;
    case M_QUAD: quad_dpar(z, d); break;
  }
}

// Running cost f0 = sum_k q_k (x_k - xref_k(t))^2 + sum_i r_i (u_i - uref_i)^2 at node time t,
// with the state reference xref_k(t) = xref_k + xslope_k t + xamp_k sin(xfreq_k t) (a constant
// reference when the three arrays are absent).
inline double xref_at(const Prob& P, int k, double t) {
  double r = P.xref[k];
  if (P.xslope) r = r + P.xslope[k] * t;
  if (P.xamp && P.xfreq) r = r + P.xamp[k] * std::sin(P.xfreq[k] * t);
  return r;
}
template <class S> S cost_f0(const Prob& P, const S* z, double t) {
  S s = S(0.0);
  for (int k = 0; k < P.nx; ++k) { S d = z[k] - S(xref_at(P, k, t)); s += S(P.q[k]) * d * d; }
  for (int i = 0; i < P.nu; ++i) { S d = z[P.nx + i] - S(P.uref[i]); s += S(P.r[i]) * d * d; }
  return s;
}
template <class S> void cost_grad(const Prob& P, const S* z, double t, S* g) {
  for (int k = 0; k < P.nx; ++k) g[k] = S(2.0) * S(P.q[k]) * (z[k] - S(xref_at(P, k, t)));
  for (int i = 0; i < P.nu; ++i) g[P.nx + i] = S(2.0) * S(P.r[i]) * (z[P.nx + i] - S(P.uref[i]));
}
inline double cost_hess_diag(const Prob& P, int a) {  // d2 f0 / d z_a^2 (constant)
  return a < P.nx ? 2.0 * P.q[a] : 2.0 * P.r[a - P.nx];
}

// ---------------------------------------------------------------------------------------
// Transcription layout
// ---------------------------------------------------------------------------------------
struct Layout {
  int nx, nu, nz;
  bool euler;
  int64_t N, nun, n, m, nb, tau;   // nun: nodes with controls; tau: column of tf, or -1
  int npath, nbin;
  std::vector<int> fin;       // components with a final row, ascending
  explicit Layout(const Prob& P) {
    nx = P.nx; nu = P.nu; nz = nx + nu; N = P.N;
    if (P.has_final) {
      if (P.fin_comp) fin.assign(P.fin_comp, P.fin_comp + P.nfin);
      else for (int k = 0; k < nx; ++k) fin.push_back(k);
    }
    euler = P.scheme == 1;
    nun = euler ? N : N + 1;
    n = (int64_t)nx * (N + 1) + (int64_t)nu * nun + (P.free_tf ? 1 : 0);
    tau = P.free_tf ? n - 1 : -1;
    nb = (int64_t)nx + (int64_t)fin.size();
    npath = P.npath;
    nbin = P.nbin;
    m = nb + (int64_t)nx * N + (int64_t)npath * nun + nbin;
  }
  int64_t path_row(int p, int64_t i) const { return nb + (int64_t)nx * N + (int64_t)p * nun + i; }
  int64_t bin_row(int q) const { return nb + (int64_t)nx * N + (int64_t)npath * nun + q; }
  // column of the boundary variable v of z = (X_0, X_N)
  int64_t bin_col(int v) const { return v < nx ? colX(0, v) : colX(N, v - nx); }
  int64_t colX(int64_t j, int k) const { return k + (int64_t)nx * j; }
  int64_t colU(int64_t j, int i) const { return (int64_t)nx * (N + 1) + i + (int64_t)nu * j; }
  int64_t col(int64_t j, int v) const { return v < nx ? colX(j, v) : colU(j, v - nx); }
  int64_t defect_row(int k, int64_t j) const { return nb + (int64_t)k * N + j; }
};

// Path inequalities: value, first derivatives (support: a or l non-zero) and the diagonal
// second derivatives 2 a_v (support: a non-zero) of row p at node z.
inline bool path_in(const Prob& P, int p, int v) {
  const int nz = P.nx + P.nu;
  return P.path_a[p * nz + v] != 0.0 || P.path_l[p * nz + v] != 0.0;
}
template <class S> S path_value(const Prob& P, int p, const S* z) {
  const int nz = P.nx + P.nu;
  S c = S(0.0);
  for (int v = 0; v < nz; ++v) {
    const double av = P.path_a[p * nz + v], lv = P.path_l[p * nz + v];
    if (av != 0.0) { const S d = z[v] - S(P.path_b[p * nz + v]); c = c + S(av) * d * d; }
    if (lv != 0.0) c = c + S(lv) * z[v];
  }
  return c - S(P.path_r[p]);
}
template <class S> S path_deriv(const Prob& P, int p, int v, const S* z) {
  const int nz = P.nx + P.nu;
  const double av = P.path_a[p * nz + v], lv = P.path_l[p * nz + v];
  return S(2.0 * av) * (z[v] - S(P.path_b[p * nz + v])) + S(lv);
}

template <class S> void gather_node(const Layout& L, const S* x, int64_t j, S* z) {
  for (int v = 0; v < L.nz; ++v) z[v] = x[L.col(j, v)];
}

// path rows: values at the nodes with a control, after the defects
template <class S> void path_rows(const Prob& P, const Layout& L, const S* x, S* c) {
  std::vector<S> z(L.nz);
  for (int64_t i = 0; i < L.nun; ++i) {
    gather_node(L, x, i, z.data());
    for (int p = 0; p < L.npath; ++p) c[L.path_row(p, i)] = path_value(P, p, z.data());
  }
}

// path rows of the Jacobian (appended after the defect rows: highest rows, columns ascending)
template <class S> void path_jacobian(const Prob& P, const Layout& L, const S* x, std::vector<int64_t>& R,
                                      std::vector<int64_t>& Cc, std::vector<S>& V) {
  std::vector<S> z(L.nz);
  for (int p = 0; p < L.npath; ++p)
    for (int64_t i = 0; i < L.nun; ++i) {
      gather_node(L, x, i, z.data());
      for (int v = 0; v < L.nz; ++v)
        if (path_in(P, p, v)) { R.push_back(L.path_row(p, i)); Cc.push_back(L.col(i, v)); V.push_back(path_deriv(P, p, v, z.data())); }
    }
}

// path rows' Hessian terms of node i: y_{p,i} 2 a_{p,v} on the diagonal (v, v)
template <class S> void path_hessian(const Prob& P, const Layout& L, const S* y, int64_t i,
                                     std::map<std::pair<int, int>, S>& blk) {
  const int nz = L.nz;
  for (int p = 0; p < L.npath; ++p)
    for (int v = 0; v < nz; ++v) {
      const double av = P.path_a[p * nz + v];
      if (av == 0.0) continue;
      if (!blk.count({v, v})) blk[{v, v}] = S(0.0);
      blk[{v, v}] = blk[{v, v}] + y[L.path_row(p, i)] * S(2.0 * av);
    }
}

// Boundary inequalities on z = (X_0, X_N): value, first derivatives (support: a or l
// non-zero) and the diagonal second derivatives 2 a_v.
inline bool bin_in(const Prob& P, int q, int v) {
  const int nz = 2 * P.nx;
  return P.bin_a[q * nz + v] != 0.0 || P.bin_l[q * nz + v] != 0.0;
}
template <class S> void gather_bnd(const Layout& L, const S* x, S* z) {
  for (int v = 0; v < 2 * L.nx; ++v) z[v] = x[L.bin_col(v)];
}
template <class S> S bin_value(const Prob& P, int q, const S* z) {
  const int nz = 2 * P.nx;
  S c = S(0.0);
  for (int v = 0; v < nz; ++v) {
    const double av = P.bin_a[q * nz + v], lv = P.bin_l[q * nz + v];
    if (av != 0.0) { const S d = z[v] - S(P.bin_b[q * nz + v]); c = c + S(av) * d * d; }
    if (lv != 0.0) c = c + S(lv) * z[v];
  }
  return c - S(P.bin_r[q]);
}
template <class S> S bin_deriv(const Prob& P, int q, int v, const S* z) {
  const int nz = 2 * P.nx;
  return S(2.0 * P.bin_a[q * nz + v]) * (z[v] - S(P.bin_b[q * nz + v])) + S(P.bin_l[q * nz + v]);
}
// the boundary rows, after the path rows
template <class S> void bin_rows(const Prob& P, const Layout& L, const S* x, S* c) {
  std::vector<S> z(2 * L.nx);
  gather_bnd(L, x, z.data());
  for (int q = 0; q < L.nbin; ++q) c[L.bin_row(q)] = bin_value(P, q, z.data());
}
template <class S> void bin_jacobian(const Prob& P, const Layout& L, const S* x, std::vector<int64_t>& R,
                                     std::vector<int64_t>& Cc, std::vector<S>& V) {
  std::vector<S> z(2 * L.nx);
  gather_bnd(L, x, z.data());
  for (int q = 0; q < L.nbin; ++q)
    for (int v = 0; v < 2 * L.nx; ++v)  // X_0 columns before X_N columns: ascending
      if (bin_in(P, q, v)) { R.push_back(L.bin_row(q)); Cc.push_back(L.bin_col(v)); V.push_back(bin_deriv(P, q, v, z.data())); }
}
// State components k whose (k, k) entry a boundary inequality needs; the node Hessian block
// has one template for every node, so (k, k) is present in every node's block.
inline bool bin_diag(const Prob& P, int k) {
  const int nz = 2 * P.nx;
  for (int q = 0; q < P.nbin; ++q)
    if (P.bin_a[q * nz + k] != 0.0 || P.bin_a[q * nz + P.nx + k] != 0.0) return true;
  return false;
}
// the boundary rows' Hessian terms of node j (j = 0 or N): y_q 2 a_{q,v} on the diagonal;
// at every node the template's (k, k) keys
template <class S> void bin_hessian(const Prob& P, const Layout& L, const S* y, int64_t j,
                                    std::map<std::pair<int, int>, S>& blk) {
  for (int k = 0; k < L.nx; ++k)
    if (bin_diag(P, k) && !blk.count({k, k})) blk[{k, k}] = S(0.0);
  const int nz = 2 * L.nx;
  for (int q = 0; q < L.nbin; ++q)
    for (int k = 0; k < L.nx; ++k) {
      if (j == 0 && P.bin_a[q * nz + k] != 0.0)
        blk[{k, k}] = blk[{k, k}] + y[L.bin_row(q)] * S(2.0 * P.bin_a[q * nz + k]);
      if (j == L.N && P.bin_a[q * nz + L.nx + k] != 0.0)
        blk[{k, k}] = blk[{k, k}] + y[L.bin_row(q)] * S(2.0 * P.bin_a[q * nz + L.nx + k]);
    }
}

// Boundary cost g(X_0, X_N): value, gradient entries and the template diagonals (a squared
// term on X_{0,k} or X_{N,k} puts (k, k) in every node block, like the boundary rows).
template <class S> S bol_value(const Prob& P, const Layout& L, const S* x) {
  S g = S(0.0);
  for (int v = 0; v < 2 * L.nx; ++v) {
    const S z = x[L.bin_col(v)];
    const double av = P.bol_a[v], lv = P.bol_l[v];
    if (av != 0.0) { const S d = z - S(P.bol_b[v]); g = g + S(av) * d * d; }
    if (lv != 0.0) g = g + S(lv) * z;
  }
  return g;
}
template <class S> void bol_gradient(const Prob& P, const Layout& L, const S* x, S* g) {
  for (int v = 0; v < 2 * L.nx; ++v) {
    const double av = P.bol_a[v], lv = P.bol_l[v];
    if (av == 0.0 && lv == 0.0) continue;
    const int64_t col = L.bin_col(v);
    g[col] = g[col] + (S(2.0 * av) * (x[col] - S(P.bol_b[v])) + S(lv));
  }
}
inline bool bol_diag(const Prob& P, int k) {
  return P.has_bol && (P.bol_a[k] != 0.0 || P.bol_a[P.nx + k] != 0.0);
}
// sigma times its Hessian in node j's block (j = 0 or N), and the template keys at every node
template <class S> void bol_hessian(const Prob& P, const Layout& L, S sigma, int64_t j,
                                    std::map<std::pair<int, int>, S>& blk) {
  if (!P.has_bol) return;
  for (int k = 0; k < L.nx; ++k) {
    if (!bol_diag(P, k)) continue;
    if (!blk.count({k, k})) blk[{k, k}] = S(0.0);
    if (j == 0 && P.bol_a[k] != 0.0) blk[{k, k}] = blk[{k, k}] + sigma * S(2.0 * P.bol_a[k]);
    if (j == L.N && P.bol_a[L.nx + k] != 0.0) blk[{k, k}] = blk[{k, k}] + sigma * S(2.0 * P.bol_a[L.nx + k]);
  }
}

// step h = T / N, or tf / N with the free final time tf = x[tau]
template <class S> S step_h(const Prob& P, const Layout& L, const S* x) {
  if (L.tau >= 0) return x[L.tau] / S((double)P.N);
  return S(P.T / (double)P.N);
}

// node time t_j = j h on the uniform grid (fixed horizon; the tracking reference needs it)
inline double node_time(const Prob& P, int64_t j) { return (double)j * (P.T / (double)P.N); }

// trapezoidal weight w_j = h (interior) or h / 2 (end nodes), and omega_j = w_j / tf
template <class S> S weight(const Prob& P, S h, int64_t j) {
  return (j == 0 || j == P.N) ? h / S(2.0) : h;
}
inline double omega(const Prob& P, int64_t j) {
  return (j == 0 || j == P.N) ? 1.0 / (2.0 * (double)P.N) : 1.0 / (double)P.N;
}

template <class S> void params_of(const Prob& P, S* p) { for (int i = 0; i < 8; ++i) p[i] = S(P.par[i]); }

// Sparse matrices in COO, one entry per structural nonzero, sorted by (row, col).
template <class S> struct Coo { std::vector<int64_t> row, col; std::vector<S> val; };

// ---- Forward Euler (paper Sec. 3): defects X_{i+1} - X_i - h f(X_i, U_i), i = 0..N-1, the
// cost g(X_N) + sum_{i<N} h f0(X_i, U_i), unknowns X_0..X_N, U_0..U_{N-1}.  Row (k, i) involves
// z_i (through f) and X_{i+1,k} (identity); node i's Hessian block collects its own rows only.
// With a free final time, dc/dtf = -f_k(z_i) / N and dF/dtf = sum_{i<N} f0(z_i) / N.
template <class S> S euler_objective(const Prob& P, const S* x) {
  Layout L(P);
  const S h = step_h(P, L, x);
  std::vector<S> z(L.nz);
  Neumaier<S> acc;
  for (int64_t j = 0; j < L.N; ++j) {
    gather_node(L, x, j, z.data());
    acc.add(h * cost_f0(P, z.data(), node_time(P, j)));
  }
  if (P.mayer)
    for (int k = 0; k < L.nx; ++k) acc.add(S(P.mayer[k]) * x[L.colX(L.N, k)]);
  if (P.has_bol) acc.add(bol_value(P, L, x));
  return acc.result();
}

template <class S> void euler_constraints(const Prob& P, const S* p, const S* x, S* c) {
  Layout L(P);
  const S h = step_h(P, L, x);
  for (int k = 0; k < L.nx; ++k) c[k] = x[L.colX(0, k)];
  for (size_t i = 0; i < L.fin.size(); ++i) c[L.nx + i] = x[L.colX(L.N, L.fin[i])];
  std::vector<S> f(L.nx), z(L.nz);
  for (int64_t j = 0; j < L.N; ++j) {
    gather_node(L, x, j, z.data());
    model_f(P, p, z.data(), f.data());
    for (int k = 0; k < L.nx; ++k) c[L.defect_row(k, j)] = (x[L.colX(j + 1, k)] - x[L.colX(j, k)]) - h * f[k];
  }
  path_rows(P, L, x, c);
}

template <class S> void euler_gradient(const Prob& P, const S* x, S* g) {
  Layout L(P);
  const S h = step_h(P, L, x);
  std::vector<S> z(L.nz), gz(L.nz);
  Neumaier<S> gt;
  for (int64_t j = 0; j < L.N; ++j) {
    gather_node(L, x, j, z.data());
    cost_grad(P, z.data(), node_time(P, j), gz.data());
    for (int v = 0; v < L.nz; ++v) g[L.col(j, v)] = h * gz[v];
    if (L.tau >= 0) gt.add(cost_f0(P, z.data(), node_time(P, j)) / S((double)L.N));
  }
  for (int k = 0; k < L.nx; ++k) g[L.colX(L.N, k)] = S(P.mayer ? P.mayer[k] : 0.0);
  if (P.has_bol) bol_gradient(P, L, x, g);
  if (L.tau >= 0) g[L.tau] = gt.result();
}

template <class S> void euler_jacobian(const Prob& P, const S* p, const S* x, Coo<S>& J) {
  Layout L(P);
  const S h = step_h(P, L, x);
  std::vector<std::vector<JEnt<S>>> nodeJ((size_t)L.N);
  std::vector<S> f((size_t)L.nx * L.N), z(L.nz);
  for (int64_t j = 0; j < L.N; ++j) {
    gather_node(L, x, j, z.data());
    model_jac(P, p, z.data(), nodeJ[j]);
    model_f(P, p, z.data(), &f[(size_t)L.nx * j]);
  }
  auto emit = [&](int64_t r, int64_t c, S v) { J.row.push_back(r); J.col.push_back(c); J.val.push_back(v); };
  for (int k = 0; k < L.nx; ++k) emit(k, L.colX(0, k), S(1.0));
  for (size_t i = 0; i < L.fin.size(); ++i) emit(L.nx + (int64_t)i, L.colX(L.N, L.fin[i]), S(1.0));
  std::vector<std::pair<int64_t, S>> ent;
  for (int k = 0; k < L.nx; ++k)
    for (int64_t j = 0; j < L.N; ++j) {
      ent.clear();
      for (auto& e : nodeJ[j]) if (e.k == k) ent.push_back({L.col(j, e.v), S(0.0) - h * e.val});
      ent.push_back({L.colX(j, k), S(-1.0)});
      ent.push_back({L.colX(j + 1, k), S(1.0)});
      if (L.tau >= 0) ent.push_back({L.tau, S(0.0) - f[(size_t)L.nx * j + k] / S((double)L.N)});
      std::stable_sort(ent.begin(), ent.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
      const int64_t r = L.defect_row(k, j);
      for (size_t i = 0; i < ent.size();) {
        S v = ent[i].second;
        size_t t = i + 1;
        while (t < ent.size() && ent[t].first == ent[i].first) { v = v + ent[t].second; ++t; }
        emit(r, ent[i].first, v);
        i = t;
      }
    }
  path_jacobian(P, L, x, J.row, J.col, J.val);
}

template <class S> void euler_hessian(const Prob& P, const S* p, const S* x, const S* y, S sigma, Coo<S>& H) {
  Layout L(P);
  const S h = step_h(P, L, x);
  std::vector<S> z(L.nz), gz(L.nz);
  std::vector<HEnt<S>> he;
  std::vector<JEnt<S>> je;
  struct Trip { int64_t r, c; S v; };
  std::vector<Trip> all;
  for (int64_t j = 0; j < L.N; ++j) {
    gather_node(L, x, j, z.data());
    he.clear();
    model_hess(P, p, z.data(), he);
    std::map<std::pair<int, int>, S> blk;
    for (int a = 0; a < L.nz; ++a)
      if (cost_hess_diag(P, a) != 0.0) blk[{a, a}] = sigma * h * S(cost_hess_diag(P, a));
    for (auto& e : he) {
      if (!blk.count({e.a, e.b})) blk[{e.a, e.b}] = S(0.0);
      blk[{e.a, e.b}] = blk[{e.a, e.b}] + y[L.defect_row(e.k, j)] * (S(0.0) - h * e.val);
    }
    path_hessian(P, L, y, j, blk);
    bol_hessian(P, L, sigma, j, blk);
    for (auto& kv : blk) all.push_back({L.col(j, kv.first.first), L.col(j, kv.first.second), kv.second});
    if (L.tau >= 0) {
      std::map<int, S> trow;
      cost_grad(P, z.data(), node_time(P, j), gz.data());
      for (int v = 0; v < L.nz; ++v)
        if (cost_hess_diag(P, v) != 0.0) trow[v] = sigma * gz[v] / S((double)L.N);
      je.clear();
      model_jac(P, p, z.data(), je);
      for (auto& e : je) {
        if (!trow.count(e.v)) trow[e.v] = S(0.0);
        trow[e.v] = trow[e.v] + y[L.defect_row(e.k, j)] * (S(0.0) - e.val / S((double)L.N));
      }
      for (auto& kv : trow) all.push_back({L.tau, L.col(j, kv.first), kv.second});
    }
  }
  std::stable_sort(all.begin(), all.end(), [](const Trip& a, const Trip& b) {
    return a.r != b.r ? a.r < b.r : a.c < b.c;
  });
  for (auto& t : all) { H.row.push_back(t.r); H.col.push_back(t.c); H.val.push_back(t.v); }
}

// Objective F = sum_j w_j f0(z_j) (trapezoidal Lagrange cost) + sum_k mayer_k X_{N,k}
template <class S> S objective(const Prob& P, const S* x) {
  if (P.scheme == 1) return euler_objective(P, x);
  Layout L(P);
  const S h = step_h(P, L, x);
  std::vector<S> z(L.nz);
  Neumaier<S> acc;
  for (int64_t j = 0; j <= L.N; ++j) {
    gather_node(L, x, j, z.data());
    acc.add(weight(P, h, j) * cost_f0(P, z.data(), node_time(P, j)));
  }
  if (P.mayer)
    for (int k = 0; k < L.nx; ++k) acc.add(S(P.mayer[k]) * x[L.colX(L.N, k)]);
  if (P.has_bol) acc.add(bol_value(P, L, x));
  return acc.result();
}

// Constraints: initial rows, final rows, then trapezoidal defects, component-major.
template <class S> void constraints(const Prob& P, const S* p, const S* x, S* c) {
  if (P.scheme == 1) return euler_constraints(P, p, x, c);
  Layout L(P);
  const S h = step_h(P, L, x);
  for (int k = 0; k < L.nx; ++k) c[k] = x[L.colX(0, k)];
  for (size_t i = 0; i < L.fin.size(); ++i) c[L.nx + i] = x[L.colX(L.N, L.fin[i])];
  std::vector<S> f((size_t)L.nx * (L.N + 1)), z(L.nz);
  for (int64_t j = 0; j <= L.N; ++j) {
    gather_node(L, x, j, z.data());
    model_f(P, p, z.data(), &f[(size_t)L.nx * j]);
  }
  for (int k = 0; k < L.nx; ++k)
    for (int64_t j = 0; j < L.N; ++j) {
      const S fj = f[(size_t)L.nx * j + k], fj1 = f[(size_t)L.nx * (j + 1) + k];
      c[L.defect_row(k, j)] = (x[L.colX(j + 1, k)] - x[L.colX(j, k)]) - h * (fj + fj1) / S(2.0);
    }
  path_rows(P, L, x, c);
  bin_rows(P, L, x, c);
}

// Gradient of F: node-local w_j grad f0, the Mayer weights at X_N, and with a free final time
// dF/dtf = sum_j omega_j f0(z_j) (the Lagrange cost is linear in tf through w_j = tf omega_j).
template <class S> void gradient(const Prob& P, const S* x, S* g) {
  if (P.scheme == 1) return euler_gradient(P, x, g);
  Layout L(P);
  const S h = step_h(P, L, x);
  std::vector<S> z(L.nz), gz(L.nz);
  Neumaier<S> gt;
  for (int64_t j = 0; j <= L.N; ++j) {
    gather_node(L, x, j, z.data());
    cost_grad(P, z.data(), node_time(P, j), gz.data());
    for (int v = 0; v < L.nz; ++v) g[L.col(j, v)] = weight(P, h, j) * gz[v];
    if (L.tau >= 0) gt.add(S(omega(P, j)) * cost_f0(P, z.data(), node_time(P, j)));
  }
  if (P.mayer)
    for (int k = 0; k < L.nx; ++k) g[L.colX(L.N, k)] = g[L.colX(L.N, k)] + S(P.mayer[k]);
  if (P.has_bol) bol_gradient(P, L, x, g);
  if (L.tau >= 0) g[L.tau] = gt.result();
}

// Jacobian in COO, one entry per structural nonzero, sorted by (row, col).

template <class S> void jacobian(const Prob& P, const S* p, const S* x, Coo<S>& J) {
  if (P.scheme == 1) return euler_jacobian(P, p, x, J);
  Layout L(P);
  const S h = step_h(P, L, x);
  // derivative entries and values of f at every node
  std::vector<std::vector<JEnt<S>>> nodeJ((size_t)L.N + 1);
  std::vector<S> f((size_t)L.nx * (L.N + 1)), z(L.nz);
  for (int64_t j = 0; j <= L.N; ++j) {
    gather_node(L, x, j, z.data());
    model_jac(P, p, z.data(), nodeJ[j]);
    model_f(P, p, z.data(), &f[(size_t)L.nx * j]);
  }
  auto emit = [&](int64_t r, int64_t c, S v) { J.row.push_back(r); J.col.push_back(c); J.val.push_back(v); };
  for (int k = 0; k < L.nx; ++k) emit(k, L.colX(0, k), S(1.0));
  for (size_t i = 0; i < L.fin.size(); ++i) emit(L.nx + (int64_t)i, L.colX(L.N, L.fin[i]), S(1.0));
  std::vector<std::pair<int64_t, S>> ent;
  for (int k = 0; k < L.nx; ++k)
    for (int64_t j = 0; j < L.N; ++j) {
      ent.clear();
      // d c_{k,j} / d z_j : -[v == x_k] - h (df_k/dz_v)(z_j) / 2
      for (auto& e : nodeJ[j]) if (e.k == k) ent.push_back({L.col(j, e.v), S(0.0) - h * e.val / S(2.0)});
      ent.push_back({L.colX(j, k), S(-1.0)});
      // d c_{k,j} / d z_{j+1} : +[v == x_k] - h (df_k/dz_v)(z_{j+1}) / 2
      for (auto& e : nodeJ[j + 1]) if (e.k == k) ent.push_back({L.col(j + 1, e.v), S(0.0) - h * e.val / S(2.0)});
      ent.push_back({L.colX(j + 1, k), S(1.0)});
      // d c_{k,j} / d tf = -(f_k(z_j) + f_k(z_{j+1})) / (2N)
      if (L.tau >= 0)
        ent.push_back({L.tau, S(0.0) - (f[(size_t)L.nx * j + k] + f[(size_t)L.nx * (j + 1) + k]) / S(2.0 * (double)L.N)});
      std::stable_sort(ent.begin(), ent.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
      const int64_t r = L.defect_row(k, j);
      for (size_t i = 0; i < ent.size();) {
        S v = ent[i].second;
        size_t t = i + 1;
        while (t < ent.size() && ent[t].first == ent[i].first) { v = v + ent[t].second; ++t; }
        emit(r, ent[i].first, v);
        i = t;
      }
    }
  path_jacobian(P, L, x, J.row, J.col, J.val);
  bin_jacobian(P, L, x, J.row, J.col, J.val);
}

// Lagrangian Hessian sigma * Hess F + sum_r y_r Hess c_r, lower triangle, sorted by (row, col).
// Boundary rows are linear.  The defect row (k, j) involves only z_j and z_{j+1}, so the
// block of node j collects the rows (k, j-1) and (k, j), each through -h/2 Hess f_k(z_j).
// With a free final time tf the last row couples tf to every node: d2 L / dtf dz_{j,v} =
// sigma omega_j df0/dz_v - 1/(2N) sum_k ybar_{j,k} df_k/dz_v (c and F are linear in tf, so
// there is no (tf, tf) entry); its structural columns are those of the model's Jacobian
// entries and of the non-zero cost weights.
template <class S> void hessian(const Prob& P, const S* p, const S* x, const S* y, S sigma, Coo<S>& H) {
  if (P.scheme == 1) return euler_hessian(P, p, x, y, sigma, H);
  Layout L(P);
  const S h = step_h(P, L, x);
  std::vector<S> z(L.nz), gz(L.nz);
  std::vector<HEnt<S>> he;
  std::vector<JEnt<S>> je;
  struct Trip { int64_t r, c; S v; };
  std::vector<Trip> all;
  for (int64_t j = 0; j <= L.N; ++j) {
    gather_node(L, x, j, z.data());
    he.clear();
    model_hess(P, p, z.data(), he);
    std::map<std::pair<int, int>, S> blk;
    for (int a = 0; a < L.nz; ++a)
      if (cost_hess_diag(P, a) != 0.0) blk[{a, a}] = S(0.0);
    for (auto& e : he) blk[{e.a, e.b}] = S(0.0);
    // sigma * w_j * Hess f0
    for (int a = 0; a < L.nz; ++a)
      if (cost_hess_diag(P, a) != 0.0) blk[{a, a}] = blk[{a, a}] + sigma * weight(P, h, j) * S(cost_hess_diag(P, a));
    // sum over the defect rows that touch node j
    for (auto& e : he) {
      if (j >= 1) {
        const S yr = y[L.defect_row(e.k, j - 1)];
        blk[{e.a, e.b}] = blk[{e.a, e.b}] + yr * (S(0.0) - h * e.val / S(2.0));
      }
      if (j <= L.N - 1) {
        const S yr = y[L.defect_row(e.k, j)];
        blk[{e.a, e.b}] = blk[{e.a, e.b}] + yr * (S(0.0) - h * e.val / S(2.0));
      }
    }
    path_hessian(P, L, y, j, blk);
    bin_hessian(P, L, y, j, blk);
    bol_hessian(P, L, sigma, j, blk);
    for (auto& kv : blk) all.push_back({L.col(j, kv.first.first), L.col(j, kv.first.second), kv.second});
    if (L.tau >= 0) {
      std::map<int, S> trow;
      cost_grad(P, z.data(), node_time(P, j), gz.data());
      for (int v = 0; v < L.nz; ++v)
        if (cost_hess_diag(P, v) != 0.0) trow[v] = sigma * S(omega(P, j)) * gz[v];
      je.clear();
      model_jac(P, p, z.data(), je);
      for (auto& e : je) {
        S yb = S(0.0);
        if (j >= 1) yb = yb + y[L.defect_row(e.k, j - 1)];
        if (j <= L.N - 1) yb = yb + y[L.defect_row(e.k, j)];
        if (!trow.count(e.v)) trow[e.v] = S(0.0);
        trow[e.v] = trow[e.v] + yb * (S(0.0) - e.val / S(2.0 * (double)L.N));
      }
      for (auto& kv : trow) all.push_back({L.tau, L.col(j, kv.first), kv.second});
    }
  }
  std::stable_sort(all.begin(), all.end(), [](const Trip& a, const Trip& b) {
    return a.r != b.r ? a.r < b.r : a.c < b.c;
  });
  for (auto& t : all) { H.row.push_back(t.r); H.col.push_back(t.c); H.val.push_back(t.v); }
}

// Plain COO products.
template <class S> void coo_mv(const Coo<S>& A, const S* v, S* out, int64_t nout) {
  for (int64_t i = 0; i < nout; ++i) out[i] = S(0.0);
  for (size_t e = 0; e < A.val.size(); ++e) out[A.row[e]] = out[A.row[e]] + A.val[e] * v[A.col[e]];
}
template <class S> void coo_mtv(const Coo<S>& A, const S* w, S* out, int64_t nout) {
  for (int64_t i = 0; i < nout; ++i) out[i] = S(0.0);
  for (size_t e = 0; e < A.val.size(); ++e) out[A.col[e]] = out[A.col[e]] + A.val[e] * w[A.row[e]];
}
template <class S> void coo_symv_lower(const Coo<S>& A, const S* v, S* out, int64_t nout) {
  for (int64_t i = 0; i < nout; ++i) out[i] = S(0.0);
  for (size_t e = 0; e < A.val.size(); ++e) {
    out[A.row[e]] = out[A.row[e]] + A.val[e] * v[A.col[e]];
    if (A.row[e] != A.col[e]) out[A.col[e]] = out[A.col[e]] + A.val[e] * v[A.row[e]];
  }
}

// (dc/dp_i)^T w for every dynamics parameter i.  Only the defect rows depend on p:
//   dc_{k,j}/dp_i = -h (df_k/dp_i(z_j) + df_k/dp_i(z_{j+1})) / 2   (Euler: -h df_k/dp_i(z_j)),
// and each sum runs with compensation over k, then j.
template <class S> void dpar_vjp(const Prob& P, const S* p, const S* x, const S* w, S* out) {
  Layout L(P);
  const int np = model_npar(P);
  const S h = step_h(P, L, x);
  std::vector<S> d((size_t)L.nx * np * (L.N + 1)), z(L.nz);
  for (int64_t j = 0; j < L.nun; ++j) {  // (Euler: node N has no control and no f term)
    gather_node(L, x, j, z.data());
    model_dpar(P, p, z.data(), &d[(size_t)L.nx * np * j]);
  }
  auto D = [&](int64_t j, int k, int i) { return d[((size_t)L.nx * j + k) * np + i]; };
  for (int i = 0; i < np; ++i) {
    Neumaier<S> acc;
    for (int k = 0; k < L.nx; ++k)
      for (int64_t j = 0; j < L.N; ++j) {
        const S dc = L.euler ? S(0.0) - h * D(j, k, i) : S(0.0) - h * (D(j, k, i) + D(j + 1, k, i)) / S(2.0);
        acc.add(w[L.defect_row(k, j)] * dc);
      }
    out[i] = acc.result();
  }
}

// Gradient of the Lagrangian sigma F + y^T c, from the analytic gradient and Jacobian.
template <class S> void lagrangian_grad(const Prob& P, const S* p, const S* x, const S* y, S sigma, S* out) {
  Layout L(P);
  std::vector<S> g(L.n), jty(L.n);
  gradient(P, x, g.data());
  Coo<S> J;
  jacobian(P, p, x, J);
  coo_mtv(J, y, jty.data(), L.n);
  for (int64_t i = 0; i < L.n; ++i) out[i] = sigma * g[i] + jty[i];
}

// KKT matrix of the interior-point step (paper Sec. 6: the solver assembles it in device
// buffers from the derivative values), lower triangle in COO sorted by (row, col):
//     [ H + diag(dx)        .      ]      dx_i = sigma_x_i + delta_w   (sigma_x may be absent)
//     [ J             -delta_c I  ]
// H and J are this oracle's own COO; every diagonal entry of the (1,1) block is present (added
// where H has none).
struct KEnt { int64_t r, c; double v; };
inline void kkt_assemble(const Layout& L, const Coo<double>& H, const Coo<double>& J, const double* sigma_x,
                         double delta_w, double delta_c, std::vector<KEnt>& K) {
  std::vector<char> has_diag(L.n, 0);
  for (size_t e = 0; e < H.val.size(); ++e) {
    double v = H.val[e];
    if (H.row[e] == H.col[e]) {
      has_diag[H.row[e]] = 1;
      v = v + ((sigma_x ? sigma_x[H.row[e]] : 0.0) + delta_w);
    }
    K.push_back({H.row[e], H.col[e], v});
  }
  for (int64_t i = 0; i < L.n; ++i)
    if (!has_diag[i]) K.push_back({i, i, (sigma_x ? sigma_x[i] : 0.0) + delta_w});
  for (size_t e = 0; e < J.val.size(); ++e) K.push_back({L.n + J.row[e], J.col[e], J.val[e]});
  for (int64_t r = 0; r < L.m; ++r) K.push_back({L.n + r, L.n + r, -delta_c});
  std::stable_sort(K.begin(), K.end(), [](const KEnt& a, const KEnt& b) { return a.r != b.r ? a.r < b.r : a.c < b.c; });
}

int check(const Prob& P) {
  if (P.N < 1 || !(P.T > 0.0)) return 2;
  if (P.scheme != 0 && P.scheme != 1) return 2;
  if (P.npath < 0 || (P.npath > 0 && (!P.path_a || !P.path_b || !P.path_l || !P.path_r))) return 2;
  if (P.nbin < 0 || (P.nbin > 0 && (!P.bin_a || !P.bin_b || !P.bin_l || !P.bin_r))) return 2;
  if (P.nbin > 0 && P.scheme == 1) return 2;  // boundary inequalities: trapezoidal scheme only
  if (P.has_bol && (!P.bol_a || !P.bol_b || !P.bol_l)) return 2;
  if (P.has_bol && P.scheme == 1)  // Euler: node N has no Hessian block, so no squared X_N term
    for (int k = 0; k < P.nx; ++k)
      if (P.bol_a[P.nx + k] != 0.0) return 2;
  // the tracking reference is tabulated at t_j = j T / N: not with a free final time
  if (P.free_tf && (P.xslope || P.xamp)) return 2;
  if (P.has_final && P.fin_comp) {
    if (P.nfin < 1 || P.nfin > P.nx) return 2;
    for (int i = 0; i < P.nfin; ++i)
      if (P.fin_comp[i] < 0 || P.fin_comp[i] >= P.nx || (i > 0 && P.fin_comp[i] <= P.fin_comp[i - 1])) return 2;
  }
  switch (P.model) {
    case M_VDP: return (P.nx == 2 && P.nu == 1) ? 0 : 2;
    case M_CARTPOLE: return (P.nx == 4 && P.nu == 1) ? 0 : 2;
    case M_HEAT: return (P.nx >= 2 && P.nu == 1 && (int)P.par[0] == P.nx) ? 0 : 2;
    case M_DINT: return (P.nx == 2 && P.nu == 1) ? 0 : 2;
    case M_QUAD: return (P.nx == 9 && P.nu == 4) ? 0 : 2;
    case M_GODDARD: return (P.nx == 3 && P.nu == 1) ? 0 : 2;
    default: return 6;
  }
}

template <class S> std::vector<S> lift(const double* a, int64_t n) {
  std::vector<S> v(n);
  for (int64_t i = 0; i < n; ++i) v[i] = S(a[i]);
  return v;
}

}  // namespace orc

// =======================================================================================
// C interface (ctypes).  Status: 0 ok, 2 bad dimensions, 6 unknown model.
// =======================================================================================
using namespace orc;

extern "C" {

int orc_dims(const Prob* P, int64_t* n, int64_t* m, int64_t* nnzj, int64_t* nnzh) {
  int st = check(*P);
  if (st) return st;
  Layout L(*P);
  *n = L.n; *m = L.m;
  // count structure by building it at a tiny horizon is not needed: count directly
  std::vector<double> z(L.nz, 0.5), p(8);
  params_of(*P, p.data());
  std::vector<JEnt<double>> je; model_jac(*P, p.data(), z.data(), je);
  int64_t perrow = 0;
  for (int k = 0; k < L.nx; ++k) {
    // distinct columns of row k on one side: f-derivative columns plus x_k itself
    std::vector<int> cols;
    for (auto& e : je) if (e.k == k) cols.push_back(e.v);
    cols.push_back(k);
    std::sort(cols.begin(), cols.end());
    const int64_t side = (int64_t)(std::unique(cols.begin(), cols.end()) - cols.begin());
    // trapezoid: both nodes' sides; Euler: node i's side plus the identity on X_{i+1,k}
    perrow += L.euler ? side + 1 : 2 * side;
  }
  // a free final time adds one entry (the tf column) to every defect row
  *nnzj = L.nb + perrow * L.N + (L.tau >= 0 ? (int64_t)L.nx * L.N : 0);
  for (int pp = 0; pp < L.npath; ++pp)
    for (int v = 0; v < L.nz; ++v)
      if (path_in(*P, pp, v)) *nnzj += L.nun;
  for (int q = 0; q < L.nbin; ++q)
    for (int v = 0; v < 2 * L.nx; ++v)
      if (bin_in(*P, q, v)) *nnzj += 1;
  std::vector<HEnt<double>> he; model_hess(*P, p.data(), z.data(), he);
  std::vector<std::pair<int, int>> keys;
  for (int a = 0; a < L.nz; ++a) if (cost_hess_diag(*P, a) != 0.0) keys.push_back({a, a});
  for (auto& e : he) keys.push_back({e.a, e.b});
  for (int pp = 0; pp < L.npath; ++pp)
    for (int v = 0; v < L.nz; ++v)
      if (P->path_a[pp * L.nz + v] != 0.0) keys.push_back({v, v});
  for (int k = 0; k < L.nx; ++k)
    if (bin_diag(*P, k)) keys.push_back({k, k});
  for (int k = 0; k < L.nx; ++k)
    if (bol_diag(*P, k)) keys.push_back({k, k});
  std::sort(keys.begin(), keys.end());
  *nnzh = (int64_t)(std::unique(keys.begin(), keys.end()) - keys.begin()) * L.nun;
  if (L.tau >= 0) {  // the tf row: model Jacobian columns and cost columns of every node
    std::vector<int> tc;
    for (auto& e : je) tc.push_back(e.v);
    for (int a = 0; a < L.nz; ++a) if (cost_hess_diag(*P, a) != 0.0) tc.push_back(a);
    std::sort(tc.begin(), tc.end());
    *nnzh += (int64_t)(std::unique(tc.begin(), tc.end()) - tc.begin()) * L.nun;
  }
  return 0;
}

int orc_jac_structure(const Prob* P, int32_t* rows, int32_t* cols) {
  int st = check(*P);
  if (st) return st;
  Layout L(*P);
  std::vector<double> x(L.n, 0.5), p(8);
  params_of(*P, p.data());
  Coo<double> J; jacobian(*P, p.data(), x.data(), J);
  for (size_t e = 0; e < J.val.size(); ++e) { rows[e] = (int32_t)J.row[e]; cols[e] = (int32_t)J.col[e]; }
  return 0;
}

int orc_hess_structure(const Prob* P, int32_t* rows, int32_t* cols) {
  int st = check(*P);
  if (st) return st;
  Layout L(*P);
  std::vector<double> x(L.n, 0.5), y(L.m, 1.0), p(8);
  params_of(*P, p.data());
  Coo<double> H; hessian(*P, p.data(), x.data(), y.data(), 1.0, H);
  for (size_t e = 0; e < H.val.size(); ++e) { rows[e] = (int32_t)H.row[e]; cols[e] = (int32_t)H.col[e]; }
  return 0;
}

// Values (double).  Any output pointer may be null.
int orc_eval(const Prob* P, const double* x, const double* y, double sigma,
             double* f, double* c, double* g, double* jv, double* hv) {
  int st = check(*P);
  if (st) return st;
  Layout L(*P);
  std::vector<double> p(8); params_of(*P, p.data());
  if (f) *f = objective(*P, x);
  if (c) constraints(*P, p.data(), x, c);
  if (g) gradient(*P, x, g);
  if (jv) { Coo<double> J; jacobian(*P, p.data(), x, J); std::copy(J.val.begin(), J.val.end(), jv); }
  if (hv) { Coo<double> H; hessian(*P, p.data(), x, y, sigma, H); std::copy(H.val.begin(), H.val.end(), hv); }
  return 0;
}

// Running-error magnitudes of the same outputs (the tolerance gate for cancellation).
int orc_eval_shadow(const Prob* P, const double* x, const double* y, double sigma,
                    double* f, double* c, double* g, double* jv, double* hv) {
  int st = check(*P);
  if (st) return st;
  Layout L(*P);
  std::vector<Sh> p(8); params_of(*P, p.data());
  auto X = lift<Sh>(x, L.n);
  auto Y = lift<Sh>(y, L.m);
  if (f) *f = shadow(objective(*P, X.data()));
  if (c) { std::vector<Sh> o(L.m); constraints(*P, p.data(), X.data(), o.data()); for (int64_t i = 0; i < L.m; ++i) c[i] = o[i].m; }
  if (g) { std::vector<Sh> o(L.n); gradient(*P, X.data(), o.data()); for (int64_t i = 0; i < L.n; ++i) g[i] = o[i].m; }
  if (jv) { Coo<Sh> J; jacobian(*P, p.data(), X.data(), J); for (size_t e = 0; e < J.val.size(); ++e) jv[e] = J.val[e].m; }
  if (hv) { Coo<Sh> H; hessian(*P, p.data(), X.data(), Y.data(), Sh(sigma), H); for (size_t e = 0; e < H.val.size(); ++e) hv[e] = H.val[e].m; }
  return 0;
}

// Products; `mag` (nullable) receives the running-error magnitudes.
int orc_jprod(const Prob* P, const double* x, const double* v, double* out, double* mag) {
  int st = check(*P);
  if (st) return st;
  Layout L(*P);
  { std::vector<double> p(8); params_of(*P, p.data());
    Coo<double> J; jacobian(*P, p.data(), x, J); coo_mv(J, v, out, L.m); }
  if (mag) {
    std::vector<Sh> p(8); params_of(*P, p.data());
    auto X = lift<Sh>(x, L.n); auto V = lift<Sh>(v, L.n);
    Coo<Sh> J; jacobian(*P, p.data(), X.data(), J);
    std::vector<Sh> o(L.m); coo_mv(J, V.data(), o.data(), L.m);
    for (int64_t i = 0; i < L.m; ++i) mag[i] = o[i].m;
  }
  return 0;
}

int orc_jtprod(const Prob* P, const double* x, const double* w, double* out, double* mag) {
  int st = check(*P);
  if (st) return st;
  Layout L(*P);
  { std::vector<double> p(8); params_of(*P, p.data());
    Coo<double> J; jacobian(*P, p.data(), x, J); coo_mtv(J, w, out, L.n); }
  if (mag) {
    std::vector<Sh> p(8); params_of(*P, p.data());
    auto X = lift<Sh>(x, L.n); auto W = lift<Sh>(w, L.m);
    Coo<Sh> J; jacobian(*P, p.data(), X.data(), J);
    std::vector<Sh> o(L.n); coo_mtv(J, W.data(), o.data(), L.n);
    for (int64_t i = 0; i < L.n; ++i) mag[i] = o[i].m;
  }
  return 0;
}

int orc_hprod(const Prob* P, const double* x, const double* y, double sigma, const double* v,
              double* out, double* mag) {
  int st = check(*P);
  if (st) return st;
  Layout L(*P);
  { std::vector<double> p(8); params_of(*P, p.data());
    Coo<double> H; hessian(*P, p.data(), x, y, sigma, H); coo_symv_lower(H, v, out, L.n); }
  if (mag) {
    std::vector<Sh> p(8); params_of(*P, p.data());
    auto X = lift<Sh>(x, L.n); auto Y = lift<Sh>(y, L.m); auto V = lift<Sh>(v, L.n);
    Coo<Sh> H; hessian(*P, p.data(), X.data(), Y.data(), Sh(sigma), H);
    std::vector<Sh> o(L.n); coo_symv_lower(H, V.data(), o.data(), L.n);
    for (int64_t i = 0; i < L.n; ++i) mag[i] = o[i].m;
  }
  return 0;
}

// Number of dynamics parameters with a derivative.
int orc_npar(const Prob* P) { return model_npar(*P); }

// (dc/dp)^T w for every dynamics parameter (out and mag hold orc_npar entries).
int orc_dpar_vjp_all(const Prob* P, const double* x, const double* w, double* out, double* mag) {
  int st = check(*P);
  if (st) return st;
  const int np = model_npar(*P);
  if (np == 0) return 6;
  Layout L(*P);
  { std::vector<double> p(8); params_of(*P, p.data()); dpar_vjp(*P, p.data(), x, w, out); }
  if (mag) {
    std::vector<Sh> p(8), o(np); params_of(*P, p.data());
    auto X = lift<Sh>(x, L.n); auto W = lift<Sh>(w, L.m);
    dpar_vjp(*P, p.data(), X.data(), W.data(), o.data());
    for (int i = 0; i < np; ++i) mag[i] = shadow(o[i]);
  }
  return 0;
}

// (dc/dmu)^T w for the Van der Pol model.
int orc_dpar_vjp(const Prob* P, const double* x, const double* w, double* out, double* mag) {
  if (P->model != M_VDP) return check(*P) ? check(*P) : 6;
  return orc_dpar_vjp_all(P, x, w, out, mag);
}

// Gradient of the Lagrangian (analytic), double.
int orc_lagrangian_grad(const Prob* P, const double* x, const double* y, double sigma, double* out) {
  int st = check(*P);
  if (st) return st;
  std::vector<double> p(8); params_of(*P, p.data());
  lagrangian_grad(*P, p.data(), x, y, sigma, out);
  return 0;
}

// ---- complex-step directional derivatives (Im f(x + i eps d) / eps), for the pins -------
int orc_cs_cons(const Prob* P, const double* x, const double* dx, double dmu, double eps, double* out) {
  int st = check(*P);
  if (st) return st;
  Layout L(*P);
  std::vector<Cx> X(L.n), p(8), c(L.m);
  for (int64_t i = 0; i < L.n; ++i) X[i] = Cx(x[i], eps * dx[i]);
  params_of(*P, p.data());
  p[0] = Cx(P->par[0], eps * dmu);
  constraints(*P, p.data(), X.data(), c.data());
  for (int64_t i = 0; i < L.m; ++i) out[i] = c[i].imag() / eps;
  return 0;
}

// Complex step along (dx, dp): Im c(x + i eps dx; p + i eps dp) / eps, dp of orc_npar entries.
int orc_cs_cons_p(const Prob* P, const double* x, const double* dx, const double* dp, double eps, double* out) {
  int st = check(*P);
  if (st) return st;
  Layout L(*P);
  std::vector<Cx> X(L.n), p(8), c(L.m);
  for (int64_t i = 0; i < L.n; ++i) X[i] = Cx(x[i], eps * dx[i]);
  params_of(*P, p.data());
  for (int i = 0; i < model_npar(*P); ++i) p[i] = Cx(P->par[i], eps * dp[i]);
  constraints(*P, p.data(), X.data(), c.data());
  for (int64_t i = 0; i < L.m; ++i) out[i] = c[i].imag() / eps;
  return 0;
}

int orc_cs_obj(const Prob* P, const double* x, const double* dx, double eps, double* out) {
  int st = check(*P);
  if (st) return st;
  Layout L(*P);
  std::vector<Cx> X(L.n);
  for (int64_t i = 0; i < L.n; ++i) X[i] = Cx(x[i], eps * dx[i]);
  *out = objective(*P, X.data()).imag() / eps;
  return 0;
}

int orc_cs_lagrangian_grad(const Prob* P, const double* x, const double* dx, const double* y, double sigma,
                           double eps, double* out) {
  int st = check(*P);
  if (st) return st;
  Layout L(*P);
  std::vector<Cx> X(L.n), Y(L.m), p(8), o(L.n);
  for (int64_t i = 0; i < L.n; ++i) X[i] = Cx(x[i], eps * dx[i]);
  for (int64_t i = 0; i < L.m; ++i) Y[i] = Cx(y[i], 0.0);
  params_of(*P, p.data());
  lagrangian_grad(*P, p.data(), X.data(), Y.data(), Cx(sigma, 0.0), o.data());
  for (int64_t i = 0; i < L.n; ++i) out[i] = o[i].imag() / eps;
  return 0;
}

// Complex-step of the analytic Jacobian's transpose product in the parameter direction:
// d/dmu (J^T w), used to pin the mixed second derivative.
int orc_cs_jtprod_dmu(const Prob* P, const double* x, const double* w, double eps, double* out) {
  int st = check(*P);
  if (st) return st;
  Layout L(*P);
  std::vector<Cx> X(L.n), W(L.m), p(8), o(L.n);
  for (int64_t i = 0; i < L.n; ++i) X[i] = Cx(x[i], 0.0);
  for (int64_t i = 0; i < L.m; ++i) W[i] = Cx(w[i], 0.0);
  params_of(*P, p.data());
  p[0] = Cx(P->par[0], eps);
  Coo<Cx> J; jacobian(*P, p.data(), X.data(), J);
  coo_mtv(J, W.data(), o.data(), L.n);
  for (int64_t i = 0; i < L.n; ++i) out[i] = o[i].imag() / eps;
  return 0;
}

// KKT assembly (see kkt_assemble): nnz, then structure and values (rows/cols/vals may be null).
int orc_kkt(const Prob* P, const double* x, const double* y, double sigma, const double* sigma_x, double delta_w,
            double delta_c, int64_t* nnz, int32_t* rows, int32_t* cols, double* vals) {
  int st = check(*P);
  if (st) return st;
  Layout L(*P);
  std::vector<double> p(8); params_of(*P, p.data());
  Coo<double> H, J;
  hessian(*P, p.data(), x, y, sigma, H);
  jacobian(*P, p.data(), x, J);
  std::vector<KEnt> K;
  kkt_assemble(L, H, J, sigma_x, delta_w, delta_c, K);
  if (nnz) *nnz = (int64_t)K.size();
  for (size_t e = 0; e < K.size(); ++e) {
    if (rows) rows[e] = (int32_t)K[e].r;
    if (cols) cols[e] = (int32_t)K[e].c;
    if (vals) vals[e] = K[e].v;
  }
  return 0;
}

// Model right-hand side at one node (for the physics pins).
int orc_model_f(const Prob* P, const double* z, double* f) {
  int st = check(*P);
  if (st) return st;
  std::vector<double> p(8); params_of(*P, p.data());
  model_f(*P, p.data(), z, f);
  return 0;
}

}  // extern "C"
