"""Python binding of the C-ABI (include/ocp.h): argument marshalling only.

Every computation runs in the CUDA library libocp_gb300.so; this module checks tensor
arguments (FP64, contiguous, on the handle's CUDA device), passes raw pointers and the
current torch stream, and turns non-zero statuses into exceptions.  There is no CPU
fallback: without the compiled library (or without a GPU) every evaluation raises.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from . import build as _build

MODEL_IDS = {"vdp": 1, "cartpole": 2, "heat": 3, "dint": 4, "quadrotor": 5, "goddard": 6}
STATUS = {0: "OCP_OK", 1: "OCP_EINVAL", 2: "OCP_EDIM", 3: "OCP_ENOMEM", 4: "OCP_ECUDA", 5: "OCP_EMODEL",
          6: "OCP_ETIMEOUT"}

_lib = None


class OcpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class _Dyn(C.Structure):
    _fields_ = [("model", C.c_int), ("params", C.c_void_p), ("nparams", C.c_int)]


class _Cost(C.Structure):
    _fields_ = [("kind", C.c_int), ("q", C.c_void_p), ("r", C.c_void_p), ("xref", C.c_void_p),
                ("uref", C.c_void_p)]


_P = C.c_void_p
_D = C.c_double
_I64 = C.c_int64
_SIGS = {
    "ocp_create": [C.POINTER(_Dyn), C.POINTER(_Cost), C.c_int, C.c_int, _I64, _D, C.POINTER(_P)],
    "ocp_destroy": [_P],
    "ocp_set_boundary": [_P, _P, _P],
    "ocp_set_tracking": [_P, _P, _P, _P],
    "ocp_set_free_final_time": [_P, C.c_int],
    "ocp_set_scheme": [_P, C.c_int],
    "ocp_set_path_constraints": [_P, C.c_int, _P, _P, _P, _P],
    "ocp_set_boundary_inequalities": [_P, C.c_int, _P, _P, _P, _P],
    "ocp_set_boundary_cost": [_P, _P, _P, _P],
    "ocp_jac_scatter_map": [_P, _P, _P, _P, _P],
    "ocp_start_point": [_P, _P, _P, _D, _P, _P],
    "ocp_jtprod_coo": [_P, _P, _P, _P, _P],
    "ocp_set_final_components": [_P, C.c_int, _P, _P],
    "ocp_set_terminal_cost": [_P, _P],
    "ocp_set_variable_bounds": [_P, _P, _P, _P, _P, _D, _D],
    "ocp_kkt_dims": [_P, C.POINTER(_I64)],
    "ocp_kkt_structure": [_P, _P, _P, _P],
    "ocp_kkt_values": [_P, _P, _P, _P, _D, _D, _P, _P],
    "ocp_dims": [_P, C.POINTER(_I64), C.POINTER(_I64), C.POINTER(_I64), C.POINTER(_I64)],
    "ocp_bounds": [_P, _P, _P, _P, _P],
    "eval_obj": [_P, _P, _P, _P],
    "eval_cons": [_P, _P, _P, _P],
    "eval_grad": [_P, _P, _P, _P],
    "jac_coo_structure": [_P, _P, _P, _P],
    "jac_coo_values": [_P, _P, _P, _P],
    "hess_coo_structure": [_P, _P, _P, _P],
    "hess_coo_values": [_P, _P, _P, _D, _P, _P],
    "jprod": [_P, _P, _P, _P, _P],
    "jtprod": [_P, _P, _P, _P, _P],
    "hprod": [_P, _P, _P, _D, _P, _P, _P],
    "ocp_eval_all": [_P, _P, _P, _D, _P, _P, _P, _P, _P, _P],
    "ocp_eval_step": [_P, _P, _P, _D, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P],
    "ocp_eval_step_host": [_P, _P, _P, _D, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P],
    "ocp_eval_step_host_async": [_P, _P, _P, _D, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P],
    "ocp_host_step_wait": [_P, _P],
    "ocp_eval_all_range": [_P, _I64, _I64, _P, _P, _D, _P, _P, _P, _P, _P, _P],
    "ocp_eval_step_range": [_P, _I64, _I64, _P, _P, _D, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P],
    "ocp_vjp_param_range": [_P, _I64, _I64, _P, _P, _P, _P, _P],
    "ocp_sum_ordered": [_P, C.c_int, _P, _P],
    "ocp_value_layout": [_P, C.POINTER(_I64), _P, C.POINTER(C.c_int32), C.POINTER(C.c_int32)],
    "ocp_vjp_param": [_P, _P, _P, _P, _P, _P],
    "ocp_eval_cons_p": [_P, _P, _P, _P, _P],
    "ocp_vjp_param_p": [_P, _P, _P, _P, _P, _P, _P],
    "ocp_set_param0": [_P, _D],
    "ocp_param_count": [_P, _P],
    "ocp_set_params": [_P, _P, C.c_int],
    "ocp_bind_params": [_P, _P],
    "ocp_vjp_params_range": [_P, _I64, _I64, _P, _P, _P, _P, _P, _P],
    "ocp_eval_cons_params": [_P, _P, _P, _P, _P],
    "ocp_vjp_params": [_P, _P, _P, _P, _P, _P, _P],
    "ocp_bind_param0": [_P, _P],
    "ocp_jprod_param": [_P, _P, _P, _P, _P, _P],
    "ocp_hprod_param": [_P, _P, _P, _D, _P, _P, _P, _P, _P],
    "ocp_eval_grad_scaled": [_P, _P, _P, _P, _P],
    "ocp_obj_hvp": [_P, _P, _P, _P, _P, _P, _P],
    "ocp_eval_obj_noalloc": [C.POINTER(_Dyn), C.POINTER(_Cost), C.c_int, C.c_int, _I64, _D, _P, _P, _P],
    "ocp_probe_fp64": [C.c_int, C.c_int, C.c_int, C.c_int, _P, _P],
    "ocp_probe_recip": [_P, _P, _I64, _P],
    "ocp_probe_sincos": [_P, _P, _P, _P, _P, _I64, _P],
    "ocp_probe_sincos_table": [_P, _P, _P, _P, _P, _I64, _P],
    "ocp_probe_exp_table": [_P, _P, _P, _I64, _P],
    "ocp_set_fault": [C.c_char_p],
    "ocp_last_error": [_P],
}


def lib():
    """Load (building first if needed) the CUDA library.  Raises if it cannot be built."""
    global _lib
    if _lib is None:
        path = os.environ.get("OCP_GB300_LIB")  # an alternative build of the same library
        if not path:
            path = _build.LIB
            if not _build.up_to_date():
                path = _build.build()
        L = C.CDLL(path)
        alt = bool(os.environ.get("OCP_GB300_LIB"))
        for name, argt in _SIGS.items():
            if alt and not hasattr(L, name):   # an older build of the library lacks newer calls
                continue
            fn = getattr(L, name)
            fn.argtypes = argt
            fn.restype = C.c_int
        L.ocp_destroy.restype = None
        L.ocp_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def probe_fp64(op, blocks, threads, iters, out, stream=None):
    """Launch the FP64 throughput probe of include/ocp_probe.h (op 0 DFMA, 1 DADD, 2 DMUL) on
    `stream`; `out` is a CUDA float64 tensor of at least blocks * threads elements.  Returns
    the number of FP64 operations the launch executes."""
    if out.dtype != torch.float64 or not out.is_cuda or out.numel() < blocks * threads:
        raise ValueError("out must be a CUDA float64 tensor of at least blocks * threads elements")
    _check(lib().ocp_probe_fp64(int(op), int(blocks), int(threads), int(iters), C.c_void_p(out.data_ptr()),
                                _stream(stream)))
    return blocks * threads * (8 * iters + 7)


def set_fault(spec: str):
    """ocp_set_fault: arm a host-side fault ("alloc:K", "upload:K", "dims"; "" disarms)."""
    _check(lib().ocp_set_fault(spec.encode()))


def probe_recip(d, out=None, stream=None):
    """ocp_probe_recip: the kernels' reciprocal of every entry of the CUDA float64 tensor d."""
    if d.dtype != torch.float64 or not d.is_cuda or not d.is_contiguous():
        raise TypeError("d must be a contiguous float64 CUDA tensor")
    out = torch.empty_like(d) if out is None else out
    _check(lib().ocp_probe_recip(C.c_void_p(d.data_ptr()), C.c_void_p(out.data_ptr()), int(d.numel()),
                                 _stream(stream)))
    return out


def probe_sincos(x, stream=None, table=False):
    """ocp_probe_sincos (or, with table=True, ocp_probe_sincos_table): (sin, cos) of the kernels'
    routine and (sin, cos) of CUDA's sincos for every entry of the CUDA float64 tensor x."""
    if x.dtype != torch.float64 or not x.is_cuda or not x.is_contiguous():
        raise TypeError("x must be a contiguous float64 CUDA tensor")
    outs = [torch.empty_like(x) for _ in range(4)]
    fn = lib().ocp_probe_sincos_table if table else lib().ocp_probe_sincos
    _check(fn(*[C.c_void_p(t.data_ptr()) for t in [x] + outs], int(x.numel()), _stream(stream)))
    return tuple(outs)


def probe_exp(x, stream=None):
    """ocp_probe_exp_table: exp of the kernels' table-driven routine and CUDA's exp for every entry
    of the CUDA float64 tensor x."""
    if x.dtype != torch.float64 or not x.is_cuda or not x.is_contiguous():
        raise TypeError("x must be a contiguous float64 CUDA tensor")
    outs = [torch.empty_like(x) for _ in range(2)]
    _check(lib().ocp_probe_exp_table(*[C.c_void_p(t.data_ptr()) for t in [x] + outs], int(x.numel()),
                                     _stream(stream)))
    return tuple(outs)


def sum_ordered(parts, out, stream=None):
    """ocp_sum_ordered: out[0] = parts[0] + parts[1] + ... in index order (CUDA float64 tensors)."""
    if parts.dtype != torch.float64 or not parts.is_cuda or not parts.is_contiguous() or parts.numel() < 1:
        raise TypeError("parts must be a non-empty contiguous float64 CUDA tensor")
    if out.dtype != torch.float64 or not out.is_cuda or out.numel() != 1:
        raise TypeError("out must be a one-element float64 CUDA tensor")
    _check(lib().ocp_sum_ordered(C.c_void_p(parts.data_ptr()), int(parts.numel()), C.c_void_p(out.data_ptr()),
                                 _stream(stream)))
    return out


_raw_stream = getattr(torch._C, "_cuda_getCurrentRawStream", None)


def _stream(stream):
    if stream is None:
        if _raw_stream is not None:   # the current stream's handle without a Stream object
            return _raw_stream(torch.cuda.current_device())
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _check(st, h=None):
    if st != 0:
        msg = lib().ocp_last_error(h)
        raise OcpError(st, msg.decode() if msg else "")


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


class OCP:
    """A transcribed optimal control problem (an `ocp_t` handle)."""

    def __init__(self, model: str, nx: int, nu: int, N: int, T: float, params, q, r, xref=None, uref=None,
                 x0=None, xf=None, xslope=None, xamp=None, xfreq=None, free_tf=False, xf_comp=None,
                 mayer=None, bounds=None, scheme="trapezoid", path=None, bineq=None, bolza=None):
        L = lib()
        self._lib = L
        self._keep = []

        def arr(v):
            if v is None:
                return None
            a = (C.c_double * len(v))(*[float(e) for e in v])
            self._keep.append(a)
            return C.cast(a, C.c_void_p)

        dyn = _Dyn(MODEL_IDS[model], arr(params) if len(params) else None, len(params))
        cost = _Cost(0, arr(q), arr(r), arr(xref), arr(uref))
        h = C.c_void_p()
        _check(L.ocp_create(C.byref(dyn), C.byref(cost), nx, nu, int(N), float(T), C.byref(h)))
        self.h = h
        self.model, self.nx, self.nu, self.N, self.T = model, nx, nu, int(N), float(T)
        if xf_comp is not None:   # final rows on the listed components, values xf
            _check(L.ocp_set_boundary(h, arr(x0), None), h)
            comps = (C.c_int32 * len(xf_comp))(*[int(k) for k in xf_comp])
            self._keep.append(comps)
            _check(L.ocp_set_final_components(h, len(xf_comp), C.cast(comps, C.c_void_p), arr(xf)), h)
        elif x0 is not None or xf is not None:
            _check(L.ocp_set_boundary(h, arr(x0), arr(xf)), h)
        if scheme != "trapezoid":
            _check(L.ocp_set_scheme(h, {"trapezoid": 0, "euler": 1}[scheme]), h)
        if path:
            self.set_path_constraints(path, _dims=False)
        if bineq:  # rows sum_v [a (z_v - b)^2 + l z_v] - r <= 0 over z = (X_0, X_N)
            flat = lambda rows: [float(v) for row in rows for v in row]
            _check(L.ocp_set_boundary_inequalities(h, len(bineq["r"]), arr(flat(bineq["a"])), arr(flat(bineq["b"])),
                                                   arr(flat(bineq["l"])), arr(bineq["r"])), h)
        if bolza:  # F += sum_v [a (z_v - b)^2 + l z_v] over z = (X_0, X_N)
            _check(L.ocp_set_boundary_cost(h, arr(bolza["a"]), arr(bolza["b"]), arr(bolza["l"])), h)
        if free_tf:
            _check(L.ocp_set_free_final_time(h, 1), h)
        if mayer is not None:
            _check(L.ocp_set_terminal_cost(h, arr(mayer)), h)
        if bounds is not None:
            b = bounds
            _check(L.ocp_set_variable_bounds(h, arr(b.get("xlo")), arr(b.get("xhi")), arr(b.get("ulo")),
                                             arr(b.get("uhi")), float(b.get("tflo", -float("inf"))),
                                             float(b.get("tfhi", float("inf")))), h)
        if xslope is not None or xamp is not None or xfreq is not None:
            # time-varying state reference xref_k + xslope_k t + xamp_k sin(xfreq_k t)
            _check(L.ocp_set_tracking(h, arr(xslope), arr(xamp), arr(xfreq)), h)
        n, m, nj, nh = _I64(), _I64(), _I64(), _I64()
        _check(L.ocp_dims(h, C.byref(n), C.byref(m), C.byref(nj), C.byref(nh)), h)
        self.n, self.m, self.nnzj, self.nnzh = n.value, m.value, nj.value, nh.value
        self.device = torch.device("cuda", torch.cuda.current_device())

    def set_path_constraints(self, path, _dims=True):
        """ocp_set_path_constraints: rows sum_v [a (z_v - b)^2 + l z_v] - r <= 0 at every node
        (path = dict of a, b, l: one list per row over z = (X_i, U_i); r: one value per row)."""
        keep = []

        def arr(v):
            a = (C.c_double * len(v))(*[float(e) for e in v])
            keep.append(a)
            return C.cast(a, C.c_void_p)

        flat = lambda rows: [float(v) for row in rows for v in row]
        _check(lib().ocp_set_path_constraints(self.h, len(path["r"]), arr(flat(path["a"])), arr(flat(path["b"])),
                                              arr(flat(path["l"])), arr(path["r"])), self.h)
        if _dims:
            n, m, nj, nh = _I64(), _I64(), _I64(), _I64()
            _check(lib().ocp_dims(self.h, C.byref(n), C.byref(m), C.byref(nj), C.byref(nh)), self.h)
            self.n, self.m, self.nnzj, self.nnzh = n.value, m.value, nj.value, nh.value

    @classmethod
    def from_workload(cls, w: dict) -> "OCP":
        return cls(w["model"], w["nx"], w["nu"], w["N"], w["T"], w["params"], w["q"], w["r"], w.get("xref"),
                   w.get("uref"), w.get("x0"), w.get("xf"), w.get("xslope"), w.get("xamp"), w.get("xfreq"),
                   bool(w.get("free_tf")), w.get("xf_comp"), w.get("mayer"), w.get("bounds"),
                   w.get("scheme", "trapezoid"), w.get("path"), w.get("bineq"), w.get("bolza"))

    def close(self):
        if getattr(self, "h", None):
            lib().ocp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- argument checks --------------------------------------------------------------
    def _vec(self, t, size, name):
        if t is None:
            raise ValueError("%s is required" % name)
        if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
            raise TypeError("%s must be a contiguous float64 CUDA tensor" % name)
        if t.numel() != size:
            raise ValueError("%s has %d elements, expected %d" % (name, t.numel(), size))
        return t

    def _out(self, t, size, name):
        if t is None:
            return torch.empty(size, dtype=torch.float64, device=self.device)
        return self._vec(t, size, name)

    # ---- C-ABI calls ------------------------------------------------------------------
    def bounds(self):
        import numpy as np
        lv, uv, lc, uc = (np.empty(self.n), np.empty(self.n), np.empty(self.m), np.empty(self.m))
        _check(lib().ocp_bounds(self.h, lv.ctypes.data_as(_P), uv.ctypes.data_as(_P), lc.ctypes.data_as(_P),
                                uc.ctypes.data_as(_P)), self.h)
        return lv, uv, lc, uc

    def eval_obj(self, x, out=None, stream=None):
        x = self._vec(x, self.n, "x")
        out = self._out(out, 1, "f")
        _check(lib().eval_obj(self.h, _ptr(x), _ptr(out), _stream(stream)), self.h)
        return out

    def eval_cons(self, x, out=None, stream=None):
        x = self._vec(x, self.n, "x")
        out = self._out(out, self.m, "c")
        _check(lib().eval_cons(self.h, _ptr(x), _ptr(out), _stream(stream)), self.h)
        return out

    def eval_grad(self, x, out=None, stream=None):
        x = self._vec(x, self.n, "x")
        out = self._out(out, self.n, "g")
        _check(lib().eval_grad(self.h, _ptr(x), _ptr(out), _stream(stream)), self.h)
        return out

    def jac_coo_structure(self, stream=None):
        rows = torch.empty(self.nnzj, dtype=torch.int32, device=self.device)
        cols = torch.empty(self.nnzj, dtype=torch.int32, device=self.device)
        _check(lib().jac_coo_structure(self.h, _ptr(rows), _ptr(cols), _stream(stream)), self.h)
        return rows, cols

    def hess_coo_structure(self, stream=None):
        rows = torch.empty(self.nnzh, dtype=torch.int32, device=self.device)
        cols = torch.empty(self.nnzh, dtype=torch.int32, device=self.device)
        _check(lib().hess_coo_structure(self.h, _ptr(rows), _ptr(cols), _stream(stream)), self.h)
        return rows, cols

    # ---- KKT matrix [H + diag(sigma_x + delta_w), J^T; J, -delta_c I] (lower triangle) -------
    def kkt_nnz(self):
        nz = _I64()
        _check(lib().ocp_kkt_dims(self.h, C.byref(nz)), self.h)
        return nz.value

    def kkt_structure(self, stream=None):
        nz = self.kkt_nnz()
        rows = torch.empty(nz, dtype=torch.int32, device=self.device)
        cols = torch.empty(nz, dtype=torch.int32, device=self.device)
        _check(lib().ocp_kkt_structure(self.h, _ptr(rows), _ptr(cols), _stream(stream)), self.h)
        return rows, cols

    def kkt_values(self, hvals, jvals, sigma_x=None, delta_w=0.0, delta_c=0.0, out=None, stream=None):
        hvals = self._vec(hvals, self.nnzh, "hvals")
        jvals = self._vec(jvals, self.nnzj, "jvals")
        if sigma_x is not None:
            sigma_x = self._vec(sigma_x, self.n, "sigma_x")
        out = self._out(out, self.kkt_nnz(), "kvals")
        _check(lib().ocp_kkt_values(self.h, _ptr(hvals), _ptr(jvals), _ptr(sigma_x), float(delta_w), float(delta_c),
                                    _ptr(out), _stream(stream)), self.h)
        return out

    def jac_coo_values(self, x, out=None, stream=None):
        x = self._vec(x, self.n, "x")
        out = self._out(out, self.nnzj, "vals")
        _check(lib().jac_coo_values(self.h, _ptr(x), _ptr(out), _stream(stream)), self.h)
        return out

    def hess_coo_values(self, x, y, sigma, out=None, stream=None):
        x = self._vec(x, self.n, "x")
        y = self._vec(y, self.m, "y")
        out = self._out(out, self.nnzh, "vals")
        _check(lib().hess_coo_values(self.h, _ptr(x), _ptr(y), float(sigma), _ptr(out), _stream(stream)), self.h)
        return out

    def jprod(self, x, v, out=None, stream=None):
        x = self._vec(x, self.n, "x")
        v = self._vec(v, self.n, "v")
        out = self._out(out, self.m, "Jv")
        _check(lib().jprod(self.h, _ptr(x), _ptr(v), _ptr(out), _stream(stream)), self.h)
        return out

    def jtprod(self, x, v, out=None, stream=None):
        x = self._vec(x, self.n, "x")
        v = self._vec(v, self.m, "v")
        out = self._out(out, self.n, "Jtv")
        _check(lib().jtprod(self.h, _ptr(x), _ptr(v), _ptr(out), _stream(stream)), self.h)
        return out

    def hprod(self, x, y, sigma, v, out=None, stream=None):
        x = self._vec(x, self.n, "x")
        y = self._vec(y, self.m, "y")
        v = self._vec(v, self.n, "v")
        out = self._out(out, self.n, "Hv")
        _check(lib().hprod(self.h, _ptr(x), _ptr(y), float(sigma), _ptr(v), _ptr(out), _stream(stream)), self.h)
        return out

    def eval_all(self, x, y, sigma, f=None, c=None, g=None, jvals=None, hvals=None, stream=None, alloc=True):
        """Fused evaluation; with alloc=True missing outputs are allocated (all five computed)."""
        x = self._vec(x, self.n, "x")
        if y is not None:
            y = self._vec(y, self.m, "y")
        if alloc:
            f = self._out(f, 1, "f"); c = self._out(c, self.m, "c"); g = self._out(g, self.n, "g")
            jvals = self._out(jvals, self.nnzj, "jvals"); hvals = self._out(hvals, self.nnzh, "hvals")
        _check(lib().ocp_eval_all(self.h, _ptr(x), _ptr(y), float(sigma), _ptr(f), _ptr(c), _ptr(g), _ptr(jvals),
                                  _ptr(hvals), _stream(stream)), self.h)
        return f, c, g, jvals, hvals

    def eval_step(self, x, y, sigma, vn, vm, outs=None, stream=None):
        """Fused step: (f, c, g, jvals, hvals, Jv, Jtv, Hv) in one pass; `outs` reuses buffers."""
        x = self._vec(x, self.n, "x"); y = self._vec(y, self.m, "y")
        vn = self._vec(vn, self.n, "vn"); vm = self._vec(vm, self.m, "vm")
        if outs is None:
            outs = (self._out(None, 1, "f"), self._out(None, self.m, "c"), self._out(None, self.n, "g"),
                    self._out(None, self.nnzj, "jvals"), self._out(None, self.nnzh, "hvals"),
                    self._out(None, self.m, "Jv"), self._out(None, self.n, "Jtv"), self._out(None, self.n, "Hv"))
        _check(lib().ocp_eval_step(self.h, _ptr(x), _ptr(y), float(sigma), _ptr(vn), _ptr(vm),
                                   *[_ptr(t) for t in outs], _stream(stream)), self.h)
        return outs

    def eval_step_range(self, node_begin, node_end, x, y, sigma, vn, vm, outs, stream=None):
        """ocp_eval_step_range: the fused step on the nodes [node_begin, node_end) only, into the
        full-size buffers `outs` = (f, c, g, jvals, hvals, Jv, Jtv, Hv); f receives the range's
        partial objective."""
        x = self._vec(x, self.n, "x"); y = self._vec(y, self.m, "y")
        vn = self._vec(vn, self.n, "vn"); vm = self._vec(vm, self.m, "vm")
        sizes = (1, self.m, self.n, self.nnzj, self.nnzh, self.m, self.n, self.n)
        names = ("f", "c", "g", "jvals", "hvals", "Jv", "Jtv", "Hv")
        outs = tuple(self._vec(o, s, nm) for o, s, nm in zip(outs, sizes, names))
        _check(lib().ocp_eval_step_range(self.h, int(node_begin), int(node_end), _ptr(x), _ptr(y), float(sigma),
                                         _ptr(vn), _ptr(vm), *[_ptr(o) for o in outs], _stream(stream)), self.h)
        return outs

    def vjp_param_range(self, node_begin, node_end, x, w, Jtw, dmu, stream=None):
        """ocp_vjp_param_range: J^T w on the nodes [node_begin, node_end) and their share of
        (dc/dmu)^T w (Van der Pol)."""
        x = self._vec(x, self.n, "x"); w = self._vec(w, self.m, "w")
        Jtw = self._vec(Jtw, self.n, "Jtw"); dmu = self._vec(dmu, 1, "dmu")
        _check(lib().ocp_vjp_param_range(self.h, int(node_begin), int(node_end), _ptr(x), _ptr(w), _ptr(Jtw),
                                         _ptr(dmu), _stream(stream)), self.h)
        return Jtw, dmu

    def vjp_params_range(self, node_begin, node_end, x, w, Jtw, dp, p=None, stream=None):
        """ocp_vjp_params_range: J^T w on the nodes [node_begin, node_end) and their shares of
        (dc/dp)^T w for every dynamics parameter."""
        x = self._vec(x, self.n, "x"); w = self._vec(w, self.m, "w"); p = self._pvec(p)
        Jtw = self._vec(Jtw, self.n, "Jtw"); dp = self._vec(dp, self.nparams, "dp")
        _check(lib().ocp_vjp_params_range(self.h, int(node_begin), int(node_end), _ptr(x), _ptr(w), _ptr(p),
                                          _ptr(Jtw), _ptr(dp), _stream(stream)), self.h)
        return Jtw, dp

    def value_layout(self):
        """ocp_value_layout: nb, values per defect row of each component, Hessian values per node
        in the X and U blocks."""
        nb, hx, hu = _I64(), C.c_int32(), C.c_int32()
        rc = (C.c_int32 * self.nx)()
        _check(lib().ocp_value_layout(self.h, C.byref(nb), C.cast(rc, _P), C.byref(hx), C.byref(hu)), self.h)
        return dict(nx=self.nx, nu=self.nu, N=self.N, nb=nb.value, has_final=nb.value > self.nx,
                    jcount=[int(v) for v in rc], hx=hx.value, hu=hu.value)

    def _hvec(self, t, size, name):
        if t is None:
            raise ValueError("%s is required" % name)
        if t.dtype != torch.float64 or t.is_cuda or not t.is_contiguous():
            raise TypeError("%s must be a contiguous float64 CPU tensor (pinned for overlapped copies)" % name)
        if t.numel() != size:
            raise ValueError("%s has %d elements, expected %d" % (name, t.numel(), size))
        return t

    def eval_step_host(self, x, y, sigma, vn, vm, outs=None, stream=None, wait=True):
        """The fused step with host (CPU) tensors in and out, through ocp_eval_step_host: the
        library copies the inputs to its device copies, runs the step and copies the outputs
        back, on its own copy streams joined to `stream` (default: the current stream).  The
        outputs are complete once `stream` is synchronized.  With wait=False
        (ocp_eval_step_host_async) `stream` does not wait for the output copy, so the next
        step overlaps it; call host_step_wait before synchronizing and reading the outputs."""
        x = self._hvec(x, self.n, "x"); y = self._hvec(y, self.m, "y")
        vn = self._hvec(vn, self.n, "vn"); vm = self._hvec(vm, self.m, "vm")
        sizes = ((1, "f"), (self.m, "c"), (self.n, "g"), (self.nnzj, "jvals"), (self.nnzh, "hvals"),
                 (self.m, "Jv"), (self.n, "Jtv"), (self.n, "Hv"))
        if outs is None:
            outs = tuple(torch.empty(k, dtype=torch.float64).pin_memory() for k, _ in sizes)
        outs = tuple(self._hvec(t, k, nm) for t, (k, nm) in zip(outs, sizes))
        fn = lib().ocp_eval_step_host if wait else lib().ocp_eval_step_host_async
        _check(fn(self.h, _ptr(x), _ptr(y), float(sigma), _ptr(vn), _ptr(vm),
                  *[_ptr(t) for t in outs], _stream(stream)), self.h)
        return outs

    def host_step_wait(self, stream=None):
        """Make `stream` wait for the output copies of every earlier host step on this handle."""
        _check(lib().ocp_host_step_wait(self.h, _stream(stream)), self.h)

    def start_point(self, xs=None, us=None, tf=0.0, out=None, stream=None):
        """x with X_{j,k} = xs[k], U_{j,i} = us[i] at every node (and tf), on the device."""
        out = self._out(out, self.n, "x")
        ax = None if xs is None else (C.c_double * self.nx)(*[float(t) for t in xs])
        au = None if us is None else (C.c_double * self.nu)(*[float(t) for t in us])
        px = None if ax is None else C.cast(ax, C.c_void_p)
        pu = None if au is None else C.cast(au, C.c_void_p)
        _check(lib().ocp_start_point(self.h, px, pu, float(tf), _ptr(out), _stream(stream)), self.h)
        return out

    def jac_scatter_map(self, stream=None):
        """(colptr, rows, slots): the Jacobian's COO in column order (int32 CUDA tensors)."""
        colptr = torch.empty(self.n + 1, dtype=torch.int32, device=self.device)
        rows = torch.empty(max(self.nnzj, 1), dtype=torch.int32, device=self.device)
        slots = torch.empty(max(self.nnzj, 1), dtype=torch.int32, device=self.device)
        _check(lib().ocp_jac_scatter_map(self.h, _ptr(colptr), _ptr(rows), _ptr(slots), _stream(stream)), self.h)
        return colptr, rows[:self.nnzj], slots[:self.nnzj]

    def jtprod_coo(self, jvals, w, out=None, stream=None):
        """J^T w from stored Jacobian values (ocp_jtprod_coo)."""
        jvals = self._vec(jvals, self.nnzj, "jvals")
        w = self._vec(w, self.m, "w")
        out = self._out(out, self.n, "Jtw")
        _check(lib().ocp_jtprod_coo(self.h, _ptr(jvals), _ptr(w), _ptr(out), _stream(stream)), self.h)
        return out

    def eval_all_range(self, node_begin, node_end, x, y, sigma, f, c, g, jvals, hvals, stream=None):
        _check(lib().ocp_eval_all_range(self.h, int(node_begin), int(node_end), _ptr(x), _ptr(y), float(sigma),
                                        _ptr(f), _ptr(c), _ptr(g), _ptr(jvals), _ptr(hvals), _stream(stream)),
               self.h)

    def vjp_param(self, x, w, Jtw=None, dmu=None, stream=None):
        x = self._vec(x, self.n, "x")
        w = self._vec(w, self.m, "w")
        Jtw = self._out(Jtw, self.n, "Jtw")
        dmu = self._out(dmu, 1, "dmu")
        _check(lib().ocp_vjp_param(self.h, _ptr(x), _ptr(w), _ptr(Jtw), _ptr(dmu), _stream(stream)), self.h)
        return Jtw, dmu

    def eval_cons_p(self, x, p0, out=None, stream=None):
        """c(x) with params[0] (Van der Pol mu) read from the one-element CUDA tensor p0 for this
        call (ocp_eval_cons_p; p0 None: the handle's value)."""
        x = self._vec(x, self.n, "x"); p0 = self._scalar(p0, "p0")
        out = self._out(out, self.m, "c")
        _check(lib().ocp_eval_cons_p(self.h, _ptr(x), _ptr(p0), _ptr(out), _stream(stream)), self.h)
        return out

    def vjp_param_p(self, x, w, p0, Jtw=None, dmu=None, stream=None):
        """(J^T w, (dc/dmu)^T w) with mu read from the CUDA scalar p0 for this call
        (ocp_vjp_param_p)."""
        x = self._vec(x, self.n, "x"); w = self._vec(w, self.m, "w"); p0 = self._scalar(p0, "p0")
        Jtw = self._out(Jtw, self.n, "Jtw")
        dmu = self._out(dmu, 1, "dmu")
        _check(lib().ocp_vjp_param_p(self.h, _ptr(x), _ptr(w), _ptr(p0), _ptr(Jtw), _ptr(dmu), _stream(stream)),
               self.h)
        return Jtw, dmu

    def set_param0(self, value: float):
        _check(lib().ocp_set_param0(self.h, float(value)), self.h)

    @property
    def nparams(self) -> int:
        """Number of dynamics parameters with a derivative (ocp_param_count): Van der Pol 1
        (mu), cart-pole 4 (m_c, m_p, l, g), Goddard 4 (Cd, beta, Tmax, b), quadrotor 1 (g),
        the double integrator and the heat model 0."""
        if getattr(self, "_nparams", None) is None:
            n = C.c_int()
            _check(lib().ocp_param_count(self.h, C.byref(n)), self.h)
            self._nparams = n.value
        return self._nparams

    def set_params(self, values):
        """Replace the dynamics parameters (host values, ocp_set_params)."""
        a = (C.c_double * len(values))(*[float(v) for v in values])
        _check(lib().ocp_set_params(self.h, a, len(values)), self.h)

    def _pvec(self, p, name="p"):
        if p is None:
            return None
        if p.dtype != torch.float64 or not p.is_cuda or p.numel() != self.nparams or not p.is_contiguous():
            raise TypeError("%s must be a contiguous float64 CUDA tensor of %d elements" % (name, self.nparams))
        return p

    def eval_cons_params(self, x, p=None, out=None, stream=None):
        """c(x; p) with the dynamics parameters read from the CUDA tensor p for this call
        (ocp_eval_cons_params; None: the handle's values)."""
        x = self._vec(x, self.n, "x"); p = self._pvec(p)
        out = self._out(out, self.m, "c")
        _check(lib().ocp_eval_cons_params(self.h, _ptr(x), _ptr(p), _ptr(out), _stream(stream)), self.h)
        return out

    def vjp_params(self, x, w, p=None, Jtw=None, dp=None, stream=None):
        """(J^T w, (dc/dp)^T w) for every dynamics parameter, p as in eval_cons_params
        (ocp_vjp_params)."""
        x = self._vec(x, self.n, "x"); w = self._vec(w, self.m, "w"); p = self._pvec(p)
        Jtw = self._out(Jtw, self.n, "Jtw")
        dp = self._out(dp, max(self.nparams, 1), "dp")
        _check(lib().ocp_vjp_params(self.h, _ptr(x), _ptr(w), _ptr(p), _ptr(Jtw), _ptr(dp), _stream(stream)),
               self.h)
        return Jtw, dp

    def _scalar(self, t, name):
        if t is None:
            return None
        if t.dtype != torch.float64 or not t.is_cuda or t.numel() != 1 or not t.is_contiguous():
            raise TypeError("%s must be a one-element contiguous float64 CUDA tensor" % name)
        return t

    def bind_param0(self, p0):
        """Read params[0] (Van der Pol mu) from the one-element CUDA tensor p0 (None unbinds).
        Launches capture the pointer, so unbinding right after them is safe."""
        p0 = self._scalar(p0, "p0")
        _check(lib().ocp_bind_param0(self.h, _ptr(p0)), self.h)

    class _Bound:
        def __init__(self, H, p0):
            self.H, self.p0 = H, p0

        def __enter__(self):
            self.H.bind_param0(self.p0)
            return self.H

        def __exit__(self, *exc):
            self.H.bind_param0(None)
            return False

    def param0(self, p0):
        """Context manager: calls inside it read params[0] from the CUDA scalar p0."""
        return OCP._Bound(self, p0)

    def bind_params(self, p):
        """Read every dynamics parameter from the CUDA tensor p (None unbinds; ocp_bind_params)."""
        p = self._pvec(p)
        _check(lib().ocp_bind_params(self.h, _ptr(p)), self.h)

    class _BoundAll:
        def __init__(self, H, p):
            self.H, self.p = H, p

        def __enter__(self):
            self.H.bind_params(self.p)
            return self.H

        def __exit__(self, *exc):
            self.H.bind_params(None)
            return False

    def params_bound(self, p):
        """Context manager: calls inside it read the dynamics parameters from the CUDA tensor p."""
        return OCP._BoundAll(self, p)

    def jprod_param(self, x, v, s=None, out=None, stream=None):
        x = self._vec(x, self.n, "x"); v = self._vec(v, self.n, "v"); s = self._scalar(s, "s")
        out = self._out(out, self.m, "Jv")
        _check(lib().ocp_jprod_param(self.h, _ptr(x), _ptr(v), _ptr(s), _ptr(out), _stream(stream)), self.h)
        return out

    def hprod_param(self, x, y, sigma, v, s=None, out=None, dmu=None, stream=None):
        x = self._vec(x, self.n, "x"); y = self._vec(y, self.m, "y"); v = self._vec(v, self.n, "v")
        s = self._scalar(s, "s"); dmu = self._scalar(dmu, "dmu")
        out = self._out(out, self.n, "Hv")
        _check(lib().ocp_hprod_param(self.h, _ptr(x), _ptr(y), float(sigma), _ptr(v), _ptr(s), _ptr(out), _ptr(dmu),
                                     _stream(stream)), self.h)
        return out

    def eval_grad_scaled(self, x, s, out=None, stream=None):
        x = self._vec(x, self.n, "x"); s = self._scalar(s, "s")
        out = self._out(out, self.n, "g")
        _check(lib().ocp_eval_grad_scaled(self.h, _ptr(x), _ptr(s), _ptr(out), _stream(stream)), self.h)
        return out

    def obj_hvp(self, x, s, v, out=None, dot=None, stream=None):
        x = self._vec(x, self.n, "x"); s = self._scalar(s, "s"); v = self._vec(v, self.n, "v")
        dot = self._scalar(dot, "dot")
        out = self._out(out, self.n, "Hv")
        _check(lib().ocp_obj_hvp(self.h, _ptr(x), _ptr(s), _ptr(v), _ptr(out), _ptr(dot), _stream(stream)), self.h)
        return out


def ocp_create(w: dict) -> OCP:
    """Create a problem from a workload description (see synth.workload)."""
    return OCP.from_workload(w)


# C-ABI names as module-level functions (handle first, then the arguments of include/ocp.h)
def eval_obj(h: OCP, x, f=None, stream=None):
    return h.eval_obj(x, f, stream)


def eval_cons(h: OCP, x, c=None, stream=None):
    return h.eval_cons(x, c, stream)


def eval_grad(h: OCP, x, g=None, stream=None):
    return h.eval_grad(x, g, stream)


def jac_coo_structure(h: OCP, stream=None):
    return h.jac_coo_structure(stream)


def jac_coo_values(h: OCP, x, vals=None, stream=None):
    return h.jac_coo_values(x, vals, stream)


def hess_coo_structure(h: OCP, stream=None):
    return h.hess_coo_structure(stream)


def hess_coo_values(h: OCP, x, y, sigma, vals=None, stream=None):
    return h.hess_coo_values(x, y, sigma, vals, stream)


def jprod(h: OCP, x, v, Jv=None, stream=None):
    return h.jprod(x, v, Jv, stream)


def jtprod(h: OCP, x, v, Jtv=None, stream=None):
    return h.jtprod(x, v, Jtv, stream)


def hprod(h: OCP, x, y, sigma, v, Hv=None, stream=None):
    return h.hprod(x, y, sigma, v, Hv, stream)


def ocp_eval_all(h: OCP, x, y, sigma, f=None, c=None, g=None, jvals=None, hvals=None, stream=None):
    return h.eval_all(x, y, sigma, f, c, g, jvals, hvals, stream)


def library_path() -> str:
    return os.path.abspath(_build.LIB)


_BATCH_SIGS = {
    "ocp_batch_create": [C.POINTER(_P), C.c_int, C.POINTER(_P)],
    "ocp_batch_destroy": [_P],
    "ocp_batch_offsets": [_P, _P, _P, _P, _P],
    "ocp_batch_set_config": [_P, C.c_int, C.c_int, C.c_int],
    "ocp_batch_get_config": [_P, _P, _P, _P],
    "ocp_batch_eval_all": [_P, _P, _P, _D, _P, _P, _P, _P, _P, _P],
    "ocp_batch_autotune": [_P, _P, _P, _D, _P, _P, _P, _P, _P, _P, _P],
    "ocp_batch_graph_capture": [_P, _P, _P, _D, _P, _P, _P, _P, _P, _P],
    "ocp_batch_graph_launch": [_P, _P],
    "ocp_batch_last_error": [_P],
}


def _blib():
    L = lib()
    if not getattr(L, "_batch_ready", False):
        for name, argt in _BATCH_SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = argt
            fn.restype = C.c_int
        L.ocp_batch_destroy.restype = None
        L.ocp_batch_last_error.restype = C.c_char_p
        L._batch_ready = True
    return L


class OCPBatch:
    """Many problems of one model evaluated by one persistent launch (`ocp_batch_t`)."""

    def __init__(self, problems):
        import numpy as np
        L = _blib()
        self.problems = list(problems)  # keeps the handles alive
        arr = (_P * len(self.problems))(*[p.h for p in self.problems])
        b = C.c_void_p()
        _check(L.ocp_batch_create(arr, len(self.problems), C.byref(b)))
        self.b = b
        cnt = len(self.problems) + 1
        self.xoff, self.coff, self.joff, self.hoff = (np.zeros(cnt, np.int64) for _ in range(4))
        self._bcheck(L.ocp_batch_offsets(b, self.xoff.ctypes.data_as(_P), self.coff.ctypes.data_as(_P),
                                         self.joff.ctypes.data_as(_P), self.hoff.ctypes.data_as(_P)))
        self.n, self.m = int(self.xoff[-1]), int(self.coff[-1])
        self.nnzj, self.nnzh = int(self.joff[-1]), int(self.hoff[-1])
        self.count = len(self.problems)
        self.device = self.problems[0].device

    def _bcheck(self, st):
        if st != 0:
            raise OcpError(st, (_blib().ocp_batch_last_error(self.b) or b"").decode())

    def close(self):
        if getattr(self, "b", None):
            _blib().ocp_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def outputs(self):
        e = lambda k: torch.empty(k, dtype=torch.float64, device=self.device)
        return e(self.count), e(self.m), e(self.n), e(self.nnzj), e(self.nnzh)

    def set_config(self, nodes_per_thread=1, threads=128, ctas_per_sm=0):
        self._bcheck(_blib().ocp_batch_set_config(self.b, nodes_per_thread, threads, ctas_per_sm))

    def get_config(self):
        a, b_, c = C.c_int(), C.c_int(), C.c_int()
        self._bcheck(_blib().ocp_batch_get_config(self.b, C.byref(a), C.byref(b_), C.byref(c)))
        return dict(nodes_per_thread=a.value, threads=b_.value, ctas_per_sm=c.value)

    def eval_all(self, x, y, sigma, f=None, c=None, g=None, jvals=None, hvals=None, stream=None):
        self._bcheck(_blib().ocp_batch_eval_all(self.b, _ptr(x), _ptr(y), float(sigma), _ptr(f), _ptr(c), _ptr(g),
                                                _ptr(jvals), _ptr(hvals), _stream(stream)))

    def autotune(self, x, y, sigma, f=None, c=None, g=None, jvals=None, hvals=None, stream=None):
        best = C.c_double()
        self._bcheck(_blib().ocp_batch_autotune(self.b, _ptr(x), _ptr(y), float(sigma), _ptr(f), _ptr(c), _ptr(g),
                                                _ptr(jvals), _ptr(hvals), _stream(stream), C.byref(best)))
        return best.value

    def graph_capture(self, x, y, sigma, f=None, c=None, g=None, jvals=None, hvals=None, stream=None):
        self._bcheck(_blib().ocp_batch_graph_capture(self.b, _ptr(x), _ptr(y), float(sigma), _ptr(f), _ptr(c),
                                                     _ptr(g), _ptr(jvals), _ptr(hvals), _stream(stream)))

    def graph_launch(self, stream=None):
        self._bcheck(_blib().ocp_batch_graph_launch(self.b, _stream(stream)))
