"""Error paths of the library under host-side fault injection (ocp_set_fault / OCP_FAULT).

Every device allocation and every table upload of ocp_create, of the setters that rebuild the
pattern, of ocp_batch_create and of the host-step mirrors is made to fail in turn, on the host
(no GPU fault is involved).  Each failure must return the documented status with a message
that names the injection, release what the call had allocated (the device's free memory is
unchanged once the handles are destroyed), leave a handle whose setter failed refusing every
further call, and leave the library working for the next call."""
import numpy as np
import pytest
import torch

from paper_2510_03932_gb300 import synth

pytestmark = pytest.mark.gpu

ENOMEM, ECUDA, EINVAL, EDIM = 3, 4, 1, 2


@pytest.fixture(scope="module")
def ocp():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2510_03932_gb300 import ocp as M
    M.lib()
    yield M
    M.set_fault("")


def _free():
    """The device's free memory with torch's cached blocks returned (only the library's
    allocations then differ between two readings)."""
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return torch.cuda.mem_get_info()[0]


def _inject_until_success(ocp, kind, make, status):
    """Fault the K-th allocation / upload for K = 1, 2, ... until `make` succeeds; every failure
    must carry `status` and the injection mark.  Returns (number of failures, the result)."""
    fails = 0
    for k in range(1, 200):
        ocp.set_fault("%s:%d" % (kind, k))
        try:
            out = make()
        except ocp.OcpError as e:
            assert e.status == status, (kind, k, e)
            assert "injected by OCP_FAULT" in str(e), (kind, k, e)
            fails += 1
            continue
        ocp.set_fault("")
        return fails, out
    raise AssertionError("the call never succeeded")


def _workload():
    # path and boundary-inequality rows add their own tables to the allocations of create
    return synth.with_bineq(synth.with_path(synth.with_horizon(synth.workload("vdp_n1e3"), 300)))


@pytest.mark.parametrize("kind,status", [("alloc", ENOMEM), ("upload", ECUDA)])
def test_create_fails_cleanly_at_every_allocation_and_upload(ocp, kind, status):
    w = _workload()
    ocp.OCP.from_workload(w).close()   # warm-up: module load, driver pools
    free0 = _free()
    fails, H = _inject_until_success(ocp, kind, lambda: ocp.OCP.from_workload(w), status)
    assert fails >= 3, fails
    x = torch.from_numpy(synth.draw(w)["x"]).cuda()
    ref = ocp.OCP.from_workload(w)
    assert torch.equal(H.eval_cons(x), ref.eval_cons(x))   # the library still works
    H.close()
    ref.close()
    del x
    torch.cuda.empty_cache()
    assert _free() == free0


def test_dims_fault_refuses_create(ocp):
    ocp.set_fault("dims")
    with pytest.raises(ocp.OcpError) as e:
        ocp.OCP.from_workload(synth.workload("vdp_n1e3"))
    assert e.value.status == EDIM and "injected" in str(e.value)
    ocp.OCP.from_workload(synth.workload("vdp_n1e3")).close()


@pytest.mark.parametrize("kind,status", [("alloc", ENOMEM), ("upload", ECUDA), ("dims", EDIM)])
def test_failed_setter_leaves_the_handle_unusable(ocp, kind, status):
    w = synth.with_horizon(synth.workload("vdp_n1e3"), 200)
    H0 = ocp.OCP.from_workload(w)
    H0.close()
    free0 = _free()
    H = ocp.OCP.from_workload(w)
    x = torch.from_numpy(synth.draw(w)["x"]).cuda()
    ocp.set_fault("dims" if kind == "dims" else "%s:1" % kind)
    with pytest.raises(ocp.OcpError) as e:
        H.set_path_constraints(synth.with_path(w)["path"])
    assert e.value.status == status and "injected" in str(e.value)
    ocp.set_fault("")
    for call in (lambda: H.eval_obj(x), lambda: H.eval_cons(x), lambda: H.jac_coo_structure(),
                 lambda: H.set_path_constraints(synth.with_path(w)["path"])):
        with pytest.raises(ocp.OcpError) as e2:
            call()
        assert e2.value.status == EINVAL and "unusable" in str(e2.value)
    H.close()
    del x
    torch.cuda.empty_cache()
    assert _free() == free0


def test_batch_create_fails_cleanly_at_every_allocation(ocp):
    ws = [synth.with_horizon(synth.workload("cartpole_n1e5"), n) for n in (300, 517, 1000)]
    probs = [ocp.OCP.from_workload(w) for w in ws]
    ocp.OCPBatch(probs).close()
    free0 = _free()
    fails, B = _inject_until_success(ocp, "alloc", lambda: ocp.OCPBatch(probs), ENOMEM)
    assert fails >= 3, fails
    B.close()
    fails, B = _inject_until_success(ocp, "upload", lambda: ocp.OCPBatch(probs), ECUDA)
    assert fails >= 2, fails
    B.close()
    assert _free() == free0
    for P in probs:
        P.close()


def test_host_step_mirror_allocation_fault(ocp):
    w = synth.with_horizon(synth.workload("vdp_n1e3"), 500)
    d = synth.draw(w)
    H = ocp.OCP.from_workload(w)
    hin = [torch.from_numpy(d[k]).pin_memory() for k in ("x", "y", "vn", "vm")]
    sizes = (1, H.m, H.n, H.nnzj, H.nnzh, H.m, H.n, H.n)
    houts = tuple(torch.empty(k, dtype=torch.float64).pin_memory() for k in sizes)
    for k in (1, 2):
        ocp.set_fault("alloc:%d" % k)
        with pytest.raises(ocp.OcpError) as e:
            H.eval_step_host(*hin[:2], w["sigma"], *hin[2:], houts)
        assert e.value.status == ENOMEM and "injected" in str(e.value)
    ocp.set_fault("")
    H.eval_step_host(*hin[:2], w["sigma"], *hin[2:], houts)   # retries its allocation and works
    torch.cuda.synchronize()
    dev = [t.cuda() for t in hin]
    ref = H.eval_step(dev[0], dev[1], w["sigma"], dev[2], dev[3])
    for a, b in zip(houts, ref):
        assert np.array_equal(a.numpy(), b.cpu().numpy())
    H.close()


def test_failed_batch_configuration_refuses_evaluation_until_reset(ocp):
    ws = [synth.with_horizon(synth.workload("cartpole_n1e5"), n) for n in (300, 517)]
    probs = [ocp.OCP.from_workload(w) for w in ws]
    B = ocp.OCPBatch(probs)
    draws = [synth.draw(w) for w in ws]
    x = torch.from_numpy(np.concatenate([d["x"] for d in draws])).cuda()
    y = torch.from_numpy(np.concatenate([d["y"] for d in draws])).cuda()
    f, c, g, jv, hv = B.outputs()
    ocp.set_fault("upload:1")
    with pytest.raises(ocp.OcpError) as e:
        B.set_config(1, 64, 0)
    assert e.value.status == ECUDA and "injected" in str(e.value)
    with pytest.raises(ocp.OcpError) as e:
        B.eval_all(x, y, 1.0, f, c, g, jv, hv)
    assert e.value.status == EINVAL and "unusable" in str(e.value)
    B.set_config(1, 128, 0)   # a successful configuration restores it
    B.eval_all(x, y, 1.0, f, c, g, jv, hv)
    ref = probs[0].eval_all(x[B.xoff[0]:B.xoff[1]], y[B.coff[0]:B.coff[1]], 1.0)
    torch.cuda.synchronize()
    assert torch.equal(jv[B.joff[0]:B.joff[1]], ref[3])
    B.close()
    for P in probs:
        P.close()
