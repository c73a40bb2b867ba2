"""The C-ABI library loads and exports every entry point of include/ocp.h; host-side
argument validation works without a GPU (these calls fail before touching CUDA)."""
import ctypes as C
import os
import re

import pytest

from paper_2510_03932_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([a-z_][a-z0-9_]*)\s*\(", text, re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    return C.CDLL(build.build())


def test_header_declares_the_calls():
    names = declared_functions()
    for n in ["ocp_create", "eval_obj", "eval_cons", "eval_grad", "jac_coo_structure", "jac_coo_values",
              "hess_coo_structure", "hess_coo_values", "jprod", "jtprod", "hprod", "ocp_eval_all"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


class Dyn(C.Structure):
    _fields_ = [("model", C.c_int), ("params", C.c_void_p), ("nparams", C.c_int)]


class Cost(C.Structure):
    _fields_ = [("kind", C.c_int), ("q", C.c_void_p), ("r", C.c_void_p), ("xref", C.c_void_p), ("uref", C.c_void_p)]


def create(lib, model, params, nx, nu, N=10, T=1.0, kind=0):
    p = (C.c_double * max(1, len(params)))(*params)
    q = (C.c_double * 64)(*([1.0] * 64))
    r = (C.c_double * 1)(0.1)
    d = Dyn(model, C.cast(p, C.c_void_p), len(params))
    c = Cost(kind, C.cast(q, C.c_void_p), C.cast(r, C.c_void_p), None, None)
    h = C.c_void_p()
    lib.ocp_create.restype = C.c_int
    lib.ocp_create.argtypes = [C.POINTER(Dyn), C.POINTER(Cost), C.c_int, C.c_int, C.c_int64, C.c_double,
                               C.POINTER(C.c_void_p)]
    st = lib.ocp_create(C.byref(d), C.byref(c), nx, nu, N, T, C.byref(h))
    lib.ocp_last_error.restype = C.c_char_p
    lib.ocp_last_error.argtypes = [C.c_void_p]
    return st, lib.ocp_last_error(None).decode()


def test_create_rejects_bad_arguments_on_the_host(lib):
    assert create(lib, 99, [1.0], 2, 1)[0] == 5                 # OCP_EMODEL: unknown model
    assert create(lib, 1, [1.0], 3, 1)[0] == 2                  # OCP_EDIM: wrong nx (Sec. 5 dimension check)
    st, msg = create(lib, 1, [1.0], 2, 2)
    assert st == 2 and "dimension" in msg
    assert create(lib, 1, [], 2, 1)[0] == 2                     # wrong number of parameters
    assert create(lib, 2, [1, 0.1, 0.5, 9.81], 4, 1, N=0)[0] == 2  # N < 1
    assert create(lib, 1, [1.0], 2, 1, T=-1.0)[0] == 1          # OCP_EINVAL
    assert create(lib, 1, [1.0], 2, 1, kind=7)[0] == 5          # unknown cost kind
    assert create(lib, 3, [200.0], 200, 1)[0] == 2              # heat: ncell out of range
    assert create(lib, 1, [1.0], 2, 1, N=2**31)[0] == 2         # n >= 2^31 does not fit int32 COO
    # the first horizon whose Jacobian no longer fits the int32 COO interface, while n still
    # does: Van der Pol nnz_J = 2 + 10 N >= 2^31 from N = 214748365; heat-64 nnz_J = 64 + 382 N
    assert create(lib, 1, [1.0], 2, 1, N=214748365)[0] == 2
    assert create(lib, 3, [64.0], 64, 1, N=(2**31 - 64 + 381) // 382)[0] == 2
    # one node fewer passes the host checks (here it stops at the missing device instead)
    assert create(lib, 1, [1.0], 2, 1, N=214748364)[0] != 2
    assert create(lib, 3, [64.0], 64, 1, N=(2**31 - 64 + 381) // 382 - 1)[0] != 2


def test_null_handle_is_rejected(lib):
    lib.eval_obj.restype = C.c_int
    lib.eval_obj.argtypes = [C.c_void_p] * 4
    assert lib.eval_obj(None, None, None, None) == 1
    lib.ocp_host_step_wait.restype = C.c_int
    lib.ocp_host_step_wait.argtypes = [C.c_void_p] * 2
    assert lib.ocp_host_step_wait(None, None) == 1


def declared_signatures():
    """name -> list of parameter kinds ("ptr", "double", "int64", "int") from include/*.h"""
    sigs = {}
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([a-z_][a-z0-9_]*)\s*\(([^)]*)\)\s*;",
                             text, re.M):
            params = [p.strip() for p in m.group(2).split(",") if p.strip() and p.strip() != "void"]
            kinds = []
            for p in params:
                if "*" in p:
                    kinds.append("ptr")
                elif re.search(r"\bdouble\b", p):
                    kinds.append("double")
                elif re.search(r"\bint64_t\b", p):
                    kinds.append("int64")
                else:
                    kinds.append("int")
            sigs[m.group(1)] = kinds
    return sigs


def _kind(t):
    if t in (C.c_void_p, C.c_char_p) or (isinstance(t, type) and issubclass(t, C._Pointer)):
        return "ptr"
    if t is C.c_double:
        return "double"
    if t is C.c_int64:
        return "int64"
    if t in (C.c_int, C.c_int32):
        return "int"
    return "?"


def test_binding_argument_lists_match_the_header():
    """Every ctypes argument list of the Python binding has the arity and the argument kinds
    (pointer, double, int64, int) of the C declaration it binds."""
    from paper_2510_03932_gb300 import ocp as O

    decl = declared_signatures()
    tables = dict(O._SIGS)
    tables.update(O._BATCH_SIGS)
    checked = 0
    for name, argt in tables.items():
        assert name in decl, name
        assert [_kind(t) for t in argt] == decl[name], (name, [_kind(t) for t in argt], decl[name])
        checked += 1
    assert checked >= 40


def test_fault_specs_and_dims_fault_on_the_host(lib):
    """ocp_set_fault parses its spec; an armed 'dims' fault makes the next ocp_create fail in
    its pattern build (before any CUDA call) with OCP_EDIM and a message naming the injection,
    and fires only once."""
    lib.ocp_set_fault.restype = C.c_int
    lib.ocp_set_fault.argtypes = [C.c_char_p]
    lib.ocp_last_error.restype = C.c_char_p
    lib.ocp_last_error.argtypes = [C.c_void_p]
    for bad in (b"bogus", b"alloc:0", b"alloc:x", b"upload", b"alloc:-2"):
        assert lib.ocp_set_fault(bad) == 1, bad
    assert lib.ocp_set_fault(b"") == 0
    assert lib.ocp_set_fault(b"dims") == 0
    st, msg = create(lib, 1, [1.0], 2, 1)
    assert st == 2 and "injected by OCP_FAULT" in msg, msg
    # disarmed after firing: the same create no longer fails in its pattern build
    assert lib.ocp_set_fault(b"") == 0
    lib.ocp_set_fault(b"dims")
    st, msg = create(lib, 1, [1.0], 2, 1, N=-1)   # rejected by validation, before the pattern build
    assert st == 2 and "injected" not in msg, msg
    st, msg = create(lib, 1, [1.0], 2, 1)         # the armed fault fires here
    assert st == 2 and "injected by OCP_FAULT" in msg, msg
    assert lib.ocp_set_fault(b"") == 0


def test_fault_from_the_environment():
    """OCP_FAULT arms the same faults at the library's first use in a fresh process."""
    import subprocess
    import sys
    code = ("import ctypes as C, sys; sys.path.insert(0, %r)\n"
            "from paper_2510_03932_gb300 import ocp\n"
            "w = dict(model='vdp', nx=2, nu=1, N=10, T=1.0, params=[1.0], q=[1.0, 1.0], r=[1.0])\n"
            "try:\n    ocp.OCP.from_workload(w)\nexcept ocp.OcpError as e:\n    print(e.status, str(e))\n" % ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300,
                       env=dict(os.environ, OCP_FAULT="dims"))
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.startswith("2 ") and "injected by OCP_FAULT" in r.stdout, r.stdout
