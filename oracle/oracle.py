"""ctypes wrapper of the CPU oracle.

TEST INFRASTRUCTURE ONLY: the test-suite, the package smoke check and the benchmark's
CPU-baseline leg call this; the CUDA library never does.  Workloads are the plain dicts
of paper_2510_03932_gb300.synth (model name, nx, nu, N, T, params, cost weights).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

_MODEL_ID = {"vdp": 1, "cartpole": 2, "heat": 3, "dint": 4, "quadrotor": 5, "goddard": 6}


class _Prob(C.Structure):
    _fields_ = [("model", C.c_int32), ("nx", C.c_int32), ("nu", C.c_int32), ("has_final", C.c_int32),
                ("N", C.c_int64), ("T", C.c_double), ("par", C.c_double * 8), ("npar", C.c_int32),
                ("pad", C.c_int32), ("q", C.c_void_p), ("r", C.c_void_p), ("xref", C.c_void_p),
                ("uref", C.c_void_p), ("xslope", C.c_void_p), ("xamp", C.c_void_p), ("xfreq", C.c_void_p),
                ("free_tf", C.c_int32), ("nfin", C.c_int32), ("fin_comp", C.c_void_p), ("mayer", C.c_void_p),
                ("scheme", C.c_int32), ("npath", C.c_int32), ("path_a", C.c_void_p), ("path_b", C.c_void_p),
                ("path_l", C.c_void_p), ("path_r", C.c_void_p), ("nbin", C.c_int32), ("bin_a", C.c_void_p),
                ("bin_b", C.c_void_p), ("bin_l", C.c_void_p), ("bin_r", C.c_void_p), ("has_bol", C.c_int32),
                ("bol_a", C.c_void_p), ("bol_b", C.c_void_p), ("bol_l", C.c_void_p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class Problem:
    """Holds the ctypes struct and keeps its arrays alive."""

    def __init__(self, w: dict, mu: float | None = None):
        self.w = w
        self._q = np.ascontiguousarray(w["q"], dtype=np.float64)
        self._r = np.ascontiguousarray(w["r"], dtype=np.float64)
        self._xref = np.ascontiguousarray(w["xref"], dtype=np.float64)
        self._uref = np.ascontiguousarray(w["uref"], dtype=np.float64)
        # optional time-varying state reference xref_k + xslope_k t + xamp_k sin(xfreq_k t)
        self._trk = [None if w.get(k) is None else np.ascontiguousarray(w[k], dtype=np.float64)
                     for k in ("xslope", "xamp", "xfreq")]
        p = _Prob()
        p.model = _MODEL_ID[w["model"]]
        p.nx, p.nu = w["nx"], w["nu"]
        p.has_final = 1 if w.get("xf") is not None else 0
        p.N, p.T = int(w["N"]), float(w["T"])
        pars = list(w["params"])
        if mu is not None:
            pars[0] = mu
        for i, v in enumerate(pars):
            p.par[i] = v
        p.npar = len(pars)
        p.q, p.r = _ptr(self._q), _ptr(self._r)
        p.xref, p.uref = _ptr(self._xref), _ptr(self._uref)
        p.xslope, p.xamp, p.xfreq = (_ptr(a) for a in self._trk)
        # free final time, final rows on a subset of the components, linear terminal cost
        p.free_tf = 1 if w.get("free_tf") else 0
        self._fin = None
        if w.get("xf_comp") is not None:
            self._fin = np.ascontiguousarray(w["xf_comp"], dtype=np.int32)
            p.has_final, p.nfin = 1, len(self._fin)
            p.fin_comp = _ptr(self._fin)
        self._mayer = None if w.get("mayer") is None else np.ascontiguousarray(w["mayer"], dtype=np.float64)
        p.mayer = _ptr(self._mayer)
        p.scheme = {"trapezoid": 0, "euler": 1}[w.get("scheme", "trapezoid")]
        # path inequalities sum_v [a (z_v - b)^2 + l z_v] - r <= 0 (lists of rows over z = (x, u))
        self._path = None
        if w.get("path"):
            pa = w["path"]
            self._path = [np.ascontiguousarray(pa[k], dtype=np.float64) for k in ("a", "b", "l", "r")]
            p.npath = len(pa["r"])
            p.path_a, p.path_b, p.path_l, p.path_r = (_ptr(a) for a in self._path)
        # boundary inequalities sum_v [a (z_v - b)^2 + l z_v] - r <= 0 over z = (X_0, X_N)
        self._bin = None
        if w.get("bineq"):
            bi = w["bineq"]
            self._bin = [np.ascontiguousarray(bi[k], dtype=np.float64) for k in ("a", "b", "l", "r")]
            p.nbin = len(bi["r"])
            p.bin_a, p.bin_b, p.bin_l, p.bin_r = (_ptr(a) for a in self._bin)
        # boundary cost sum_v [a (z_v - b)^2 + l z_v] over z = (X_0, X_N), added to F
        self._bol = None
        if w.get("bolza"):
            bo = w["bolza"]
            self._bol = [np.ascontiguousarray(bo[k], dtype=np.float64) for k in ("a", "b", "l")]
            p.has_bol = 1
            p.bol_a, p.bol_b, p.bol_l = (_ptr(a) for a in self._bol)
        self.s = p
        n, m, nj, nh = (C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64())
        st = lib().orc_dims(C.byref(p), C.byref(n), C.byref(m), C.byref(nj), C.byref(nh))
        if st != 0:
            raise ValueError("oracle: bad problem (status %d)" % st)
        self.n, self.m, self.nnzj, self.nnzh = n.value, m.value, nj.value, nh.value

    def ref(self):
        return C.byref(self.s)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(st):
    if st != 0:
        raise RuntimeError("oracle call failed with status %d" % st)


def jac_structure(P: Problem):
    rows = np.empty(P.nnzj, np.int32); cols = np.empty(P.nnzj, np.int32)
    _check(lib().orc_jac_structure(P.ref(), _ptr(rows), _ptr(cols)))
    return rows, cols


def hess_structure(P: Problem):
    rows = np.empty(P.nnzh, np.int32); cols = np.empty(P.nnzh, np.int32)
    _check(lib().orc_hess_structure(P.ref(), _ptr(rows), _ptr(cols)))
    return rows, cols


def evaluate(P: Problem, x, y, sigma: float, shadow: bool = False) -> dict:
    """Objective, constraints, gradient, Jacobian and Hessian values (and shadows)."""
    x, y = _f64(x), _f64(y)
    f = np.zeros(1); c = np.empty(P.m); g = np.empty(P.n); jv = np.empty(P.nnzj); hv = np.empty(P.nnzh)
    _check(lib().orc_eval(P.ref(), _ptr(x), _ptr(y), C.c_double(sigma), _ptr(f), _ptr(c), _ptr(g),
                          _ptr(jv), _ptr(hv)))
    out = dict(f=f[0], c=c, g=g, jac=jv, hess=hv)
    if shadow:
        fm = np.zeros(1); cm = np.empty(P.m); gm = np.empty(P.n); jm = np.empty(P.nnzj); hm = np.empty(P.nnzh)
        _check(lib().orc_eval_shadow(P.ref(), _ptr(x), _ptr(y), C.c_double(sigma), _ptr(fm), _ptr(cm),
                                     _ptr(gm), _ptr(jm), _ptr(hm)))
        out.update(f_mag=fm[0], c_mag=cm, g_mag=gm, jac_mag=jm, hess_mag=hm)
    return out


def jprod(P, x, v, shadow=False):
    x, v = _f64(x), _f64(v)
    o = np.empty(P.m); m = np.empty(P.m) if shadow else None
    _check(lib().orc_jprod(P.ref(), _ptr(x), _ptr(v), _ptr(o), _ptr(m)))
    return (o, m) if shadow else o


def jtprod(P, x, w, shadow=False):
    x, w = _f64(x), _f64(w)
    o = np.empty(P.n); m = np.empty(P.n) if shadow else None
    _check(lib().orc_jtprod(P.ref(), _ptr(x), _ptr(w), _ptr(o), _ptr(m)))
    return (o, m) if shadow else o


def hprod(P, x, y, sigma, v, shadow=False):
    x, y, v = _f64(x), _f64(y), _f64(v)
    o = np.empty(P.n); m = np.empty(P.n) if shadow else None
    _check(lib().orc_hprod(P.ref(), _ptr(x), _ptr(y), C.c_double(sigma), _ptr(v), _ptr(o), _ptr(m)))
    return (o, m) if shadow else o


def dpar_vjp(P, x, w, shadow=False):
    x, w = _f64(x), _f64(w)
    o = np.zeros(1); m = np.zeros(1)
    _check(lib().orc_dpar_vjp(P.ref(), _ptr(x), _ptr(w), _ptr(o), _ptr(m)))
    return (o[0], m[0]) if shadow else o[0]


def npar(P) -> int:
    """Number of dynamics parameters with a derivative (Van der Pol 1, cart-pole 4, Goddard 4,
    quadrotor 1, the others 0)."""
    return int(lib().orc_npar(P.ref()))


def dpar_vjp_all(P, x, w, shadow=False):
    """(dc/dp)^T w for every dynamics parameter, with its magnitude shadow."""
    x, w = _f64(x), _f64(w)
    k = npar(P)
    o = np.zeros(k); m = np.zeros(k)
    _check(lib().orc_dpar_vjp_all(P.ref(), _ptr(x), _ptr(w), _ptr(o), _ptr(m)))
    return (o, m) if shadow else o


def lagrangian_grad(P, x, y, sigma):
    x, y = _f64(x), _f64(y)
    o = np.empty(P.n)
    _check(lib().orc_lagrangian_grad(P.ref(), _ptr(x), _ptr(y), C.c_double(sigma), _ptr(o)))
    return o


def cs_cons(P, x, dx, dmu=0.0, eps=1e-30):
    x, dx = _f64(x), _f64(dx)
    o = np.empty(P.m)
    _check(lib().orc_cs_cons(P.ref(), _ptr(x), _ptr(dx), C.c_double(dmu), C.c_double(eps), _ptr(o)))
    return o


def cs_cons_p(P, x, dx, dp, eps=1e-30):
    """Complex step of c along (dx, dp), dp with one entry per dynamics parameter."""
    x, dx, dp = _f64(x), _f64(dx), _f64(dp)
    o = np.empty(P.m)
    _check(lib().orc_cs_cons_p(P.ref(), _ptr(x), _ptr(dx), _ptr(dp), C.c_double(eps), _ptr(o)))
    return o


def cs_obj(P, x, dx, eps=1e-30):
    x, dx = _f64(x), _f64(dx)
    o = np.zeros(1)
    _check(lib().orc_cs_obj(P.ref(), _ptr(x), _ptr(dx), C.c_double(eps), _ptr(o)))
    return o[0]


def cs_lagrangian_grad(P, x, dx, y, sigma, eps=1e-30):
    x, dx, y = _f64(x), _f64(dx), _f64(y)
    o = np.empty(P.n)
    _check(lib().orc_cs_lagrangian_grad(P.ref(), _ptr(x), _ptr(dx), _ptr(y), C.c_double(sigma),
                                        C.c_double(eps), _ptr(o)))
    return o


def cs_jtprod_dmu(P, x, w, eps=1e-30):
    x, w = _f64(x), _f64(w)
    o = np.empty(P.n)
    _check(lib().orc_cs_jtprod_dmu(P.ref(), _ptr(x), _ptr(w), C.c_double(eps), _ptr(o)))
    return o


def model_f(P, z):
    z = _f64(z)
    o = np.empty(P.w["nx"])
    _check(lib().orc_model_f(P.ref(), _ptr(z), _ptr(o)))
    return o


def kkt(P, x, y, sigma, sigma_x=None, delta_w=0.0, delta_c=0.0):
    """KKT matrix [H + diag(sigma_x + delta_w), .; J, -delta_c I] (lower triangle, COO sorted)."""
    x, y = _f64(x), _f64(y)
    sx = None if sigma_x is None else _f64(sigma_x)
    nnz = C.c_int64()
    _check(lib().orc_kkt(P.ref(), _ptr(x), _ptr(y), C.c_double(sigma), _ptr(sx), C.c_double(delta_w),
                         C.c_double(delta_c), C.byref(nnz), None, None, None))
    rows = np.empty(nnz.value, np.int32); cols = np.empty(nnz.value, np.int32); vals = np.empty(nnz.value)
    _check(lib().orc_kkt(P.ref(), _ptr(x), _ptr(y), C.c_double(sigma), _ptr(sx), C.c_double(delta_w),
                         C.c_double(delta_c), None, _ptr(rows), _ptr(cols), _ptr(vals)))
    return rows, cols, vals
