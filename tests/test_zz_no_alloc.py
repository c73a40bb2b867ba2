"""ocp_eval_obj_noalloc, the objective for callers that cannot allocate device memory.

Such callers (a real-time control loop that must not allocate after start-up, a framework
whose allocator owns all device memory) get the objective from a file-scope device scratch
array instead of handle-owned scratch.  This test calls that entry point through the C-ABI
twice in a row, on two different inputs, and compares each result with the handle-based
eval_obj and with the CPU oracle's objective within the parity tolerance, for every model the entry point serves (Van der Pol,
cart-pole, heat, double integrator, quadrotor: tiles of 256, 128, 32 and 64 nodes).  After a
warm-up call (the first call on a device loads the library's kernels and looks up the
array's address) it checks that the device's free memory is the same before and after two
more calls, i.e. that the entry point allocates nothing.  It also checks that a horizon too
large for the static array is refused before any launch.  It is collected last so that a run stopping at
the first failure has run every other test first.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2510_03932_gb300 import synth

pytestmark = pytest.mark.gpu


def _entry(ocp):
    fn = ocp.lib().ocp_eval_obj_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.POINTER(ocp._Dyn), C.POINTER(ocp._Cost), C.c_int, C.c_int, C.c_int64, C.c_double,
                   C.c_void_p, C.c_void_p, C.c_void_p]
    return fn


def _desc(ocp, w, keep):
    def arr(v):
        if v is None:
            return None
        a = (C.c_double * len(v))(*[float(e) for e in v])
        keep.append(a)
        return C.cast(a, C.c_void_p)
    dyn = ocp._Dyn(ocp.MODEL_IDS[w["model"]], arr(w["params"]) if w["params"] else None, len(w["params"]))
    cost = ocp._Cost(0, arr(w["q"]), arr(w["r"]), arr(w["xref"]), arr(w["uref"]))
    return dyn, cost


CASES = [("vdp_n1e3", 1000), ("cartpole_n1e5", 5000), ("heat_n2e4", 300), ("dint", 700),
         ("quadrotor_n1e3", 3000)]


def _plain(w):
    """The workload with a constant state reference (the entry point takes the cost weights and
    the constant reference of ocp_create only)."""
    return dict(w, xslope=None, xamp=None, xfreq=None)


@pytest.mark.parametrize("name,N", CASES)
def test_noalloc_objective_matches_eval_obj_twice(name, N):
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2510_03932_gb300 import ocp
    fn = _entry(ocp)
    w = _plain(synth.with_horizon(synth.workload(name), N))
    H = ocp.OCP.from_workload(w)
    keep = []
    dyn, cost = _desc(ocp, w, keep)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    refs = []
    for call, seed in enumerate([w["seed"], w["seed"] + 77]):
        x = torch.from_numpy(synth.draw(w, seed=seed)["x"]).cuda()
        refs.append(float(H.eval_obj(x)))
        st = fn(C.byref(dyn), C.byref(cost), w["nx"], w["nu"], w["N"], w["T"], C.c_void_p(x.data_ptr()),
                C.c_void_p(out[call:call + 1].data_ptr()), stream)
        assert st == 0, ocp.lib().ocp_last_error(None)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for g, r in zip(got, refs):
        assert abs(g - r) <= 1e-12 * abs(r) + 1e-14, (g, r)
    # and against the CPU oracle's objective of the same inputs, through the parity gate
    from oracle import oracle as O
    P = O.Problem(w)
    for g, seed in zip(got, [w["seed"], w["seed"] + 77]):
        d = synth.draw(w, seed=seed)
        ev = O.evaluate(P, d["x"], d["y"], w["sigma"], shadow=True)
        assert abs(g - ev["f"]) <= 1e-12 * abs(ev["f"]) + 1e-14 or abs(g - ev["f"]) <= 1e-12 * ev["f_mag"], (g, ev["f"])
    H.close()


@pytest.mark.parametrize("name,N", CASES)
def test_noalloc_calls_leave_device_memory_unchanged(name, N):
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2510_03932_gb300 import ocp
    fn = _entry(ocp)
    w = _plain(synth.with_horizon(synth.workload(name), N))
    keep = []
    dyn, cost = _desc(ocp, w, keep)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    x = torch.from_numpy(synth.draw(w)["x"]).cuda()
    f = torch.zeros(2, dtype=torch.float64, device="cuda")
    args = (C.byref(dyn), C.byref(cost), w["nx"], w["nu"], w["N"], w["T"], C.c_void_p(x.data_ptr()))
    assert fn(*args, C.c_void_p(f[0:1].data_ptr()), stream) == 0   # warm-up: module load, address lookup
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for k in range(2):
        assert fn(*args, C.c_void_p(f[k:k + 1].data_ptr()), stream) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert float(f[0]) == float(f[1])   # same input, same reduction order: bit-identical


def test_noalloc_rejects_horizons_beyond_the_static_scratch():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2510_03932_gb300 import ocp
    fn = _entry(ocp)
    w = synth.workload("vdp_n1e3")
    keep = []
    dyn, cost = _desc(ocp, w, keep)
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    f = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = fn(C.byref(dyn), C.byref(cost), 2, 1, 65536 * 255 + 10, 10.0, C.c_void_p(x.data_ptr()),
            C.c_void_p(f.data_ptr()), None)
    assert st == 2  # OCP_EDIM, refused before any launch
    assert b"static scratch" in ocp.lib().ocp_last_error(None)
