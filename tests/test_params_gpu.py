"""Derivatives in every dynamics parameter through the C-ABI (ocp_vjp_params,
ocp_eval_cons_params, ocp_bind_params) against the oracle.

  - (dc/dp)^T w and J^T w of one launch against the oracle's dpar_vjp_all and jtprod, through the
    parity gate, at horizons spanning several tiles with a ragged tail, with and without path
    inequalities;
  - parameters read from device memory: with the handle's own values every output is bit-identical
    to the host-parameter launch (the constants are recomputed with the same arithmetic); with
    other values, c, J v, J^T w, H v and (dc/dp)^T w agree with the oracle built on those values;
  - the reductions are deterministic run to run; models without parameters and the forward Euler
    scheme are refused with OCP_EMODEL;
  - the differentiation form: gradcheck in (x, p) for the cart-pole, Goddard and quadrotor models,
    gradgradcheck in x, and a clear error for second derivatives in their parameters.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2510_03932_gb300 import synth
from parity import gate

pytestmark = pytest.mark.gpu

CASES = [("vdp_n1e3", 1000), ("cartpole_n1e5", 1000), ("cartpole_n1e5", 129), ("goddard_n1e3", 1000),
         ("quadrotor_n1e3", 700), ("cartpole_n1e5+path", 517), ("goddard_n1e3+path", 300),
         ("quadrotor_n1e3+path", 129)]


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2510_03932_gb300 import ocp
    ocp.lib()
    return ocp


def case(name, N, params=None):
    base, *plus = name.split("+")
    w = synth.with_horizon(synth.workload(base), N)
    if "path" in plus:
        w = synth.with_path(w)
    if params is not None:
        w = dict(w, params=list(params))
    return w, synth.draw(w)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def perturbed(w):
    """Other parameter values of the same model (the heat count and the double integrator have none)."""
    k = {"vdp": 1, "cartpole": 4, "goddard": 4, "quadrotor": 1}[w["model"]]
    scale = [1.13, 0.91, 1.07, 0.97][:k]
    return [p * s for p, s in zip(w["params"][:k], scale)] + list(w["params"][k:])


@pytest.mark.parametrize("name,N", CASES)
def test_vjp_params_against_oracle(M, name, N):
    w, d = case(name, N)
    H = M.OCP.from_workload(w)
    P = O.Problem(w)
    x, wv = dev(d["x"]), dev(d["vm"])
    Jtw, dp = H.vjp_params(x, wv)
    torch.cuda.synchronize()
    ref, mag = O.dpar_vjp_all(P, d["x"], d["vm"], shadow=True)
    gate("dc/dp^T w", dp.cpu().numpy(), ref, mag)
    gx, gxm = O.jtprod(P, d["x"], d["vm"], shadow=True)
    gate("J^T w", Jtw.cpu().numpy(), gx, gxm)
    # the same J^T w as the plain product (the parameter sums are extra work in the same kernel)
    assert torch.equal(Jtw, H.jtprod(x, wv))
    # deterministic: fixed-order tile sums, the same bits on every call
    Jtw2, dp2 = H.vjp_params(x, wv)
    assert torch.equal(dp, dp2) and torch.equal(Jtw, Jtw2)
    H.close()


@pytest.mark.parametrize("name,N", CASES)
def test_device_parameters_own_values_bit_identical(M, name, N):
    w, d = case(name, N)
    H = M.OCP.from_workload(w)
    x, wv = dev(d["x"]), dev(d["vm"])
    p = torch.tensor(w["params"][:H.nparams], dtype=torch.float64, device="cuda")
    assert torch.equal(H.eval_cons_params(x, p), H.eval_cons(x))
    a, b = H.vjp_params(x, wv, p), H.vjp_params(x, wv)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    vn, y = dev(d["vn"]), dev(d["y"])
    with H.params_bound(p):
        jv, hv = H.jprod(x, vn).clone(), H.hprod(x, y, 0.7, vn).clone()
    assert torch.equal(jv, H.jprod(x, vn)) and torch.equal(hv, H.hprod(x, y, 0.7, vn))
    H.close()


@pytest.mark.parametrize("name,N", CASES)
def test_device_parameters_other_values_against_oracle(M, name, N):
    w, d = case(name, N)
    H = M.OCP.from_workload(w)
    w2 = dict(w, params=perturbed(w))
    P2 = O.Problem(w2)
    x, wv, vn, y = dev(d["x"]), dev(d["vm"]), dev(d["vn"]), dev(d["y"])
    p2 = torch.tensor(w2["params"][:H.nparams], dtype=torch.float64, device="cuda")
    c = H.eval_cons_params(x, p2)
    Jtw, dp = H.vjp_params(x, wv, p2)
    with H.params_bound(p2):
        jv = H.jprod(x, vn).clone()
        hv = H.hprod(x, y, 0.7, vn).clone()
    c_host = H.eval_cons(x)   # unbound again: the handle's own values
    torch.cuda.synchronize()
    r = O.evaluate(P2, d["x"], d["y"], 0.7, shadow=True)
    gate("c(p')", c.cpu().numpy(), r["c"], r["c_mag"])
    ref, mag = O.dpar_vjp_all(P2, d["x"], d["vm"], shadow=True)
    gate("dc/dp^T w (p')", dp.cpu().numpy(), ref, mag)
    gx, gxm = O.jtprod(P2, d["x"], d["vm"], shadow=True)
    gate("J^T w (p')", Jtw.cpu().numpy(), gx, gxm)
    j, jm = O.jprod(P2, d["x"], d["vn"], shadow=True)
    gate("J v (p')", jv.cpu().numpy(), j, jm)
    hh, hm = O.hprod(P2, d["x"], d["y"], 0.7, d["vn"], shadow=True)
    gate("H v (p')", hv.cpu().numpy(), hh, hm)
    assert not torch.equal(c, c_host)
    H.close()


def test_set_params_moves_the_host_values(M):
    w, d = case("cartpole_n1e5", 300)
    H = M.OCP.from_workload(w)
    w2 = dict(w, params=perturbed(w))
    x = dev(d["x"])
    p2 = torch.tensor(w2["params"], dtype=torch.float64, device="cuda")
    c_dev = H.eval_cons_params(x, p2).clone()
    H.set_params(w2["params"])
    assert torch.equal(H.eval_cons(x), c_dev)
    with pytest.raises(M.OcpError) as e:
        H.set_params(w2["params"][:3])
    assert e.value.status == 2   # OCP_EDIM
    with pytest.raises(M.OcpError):
        H.set_params([1.0, float("nan"), 1.0, 1.0])
    H.close()


@pytest.mark.parametrize("name", ["dint", "heat_n2e4"])
def test_models_without_parameters_refuse(M, name):
    w, d = case(name, 40)
    H = M.OCP.from_workload(w)
    assert H.nparams == 0
    x, wv = dev(d["x"]), dev(d["vm"])
    with pytest.raises(M.OcpError) as e:
        H.vjp_params(x, wv)
    assert e.value.status == 5   # OCP_EMODEL
    one = torch.ones(1, dtype=torch.float64, device="cuda")
    from paper_2510_03932_gb300.ocp import lib, _ptr
    assert lib().ocp_bind_params(H.h, _ptr(one)) == 5
    assert lib().ocp_eval_cons_params(H.h, _ptr(x), _ptr(one), _ptr(torch.empty(H.m, dtype=torch.float64,
                                                                                 device="cuda")), None) == 5
    H.close()


def test_euler_scheme(M):
    """Under forward Euler the device parameters serve the constraints (checked against the
    oracle at other values); the parameter derivative and the bound products are refused."""
    w, d = case("cartpole_n1e5", 333)
    w = dict(w, scheme="euler")
    d = synth.draw(w)
    H = M.OCP.from_workload(w)
    w2 = dict(w, params=perturbed(w))
    x, wv, vn = dev(d["x"]), dev(d["vm"]), dev(d["vn"])
    p2 = torch.tensor(w2["params"], dtype=torch.float64, device="cuda")
    c = H.eval_cons_params(x, p2)
    torch.cuda.synchronize()
    r = O.evaluate(O.Problem(w2), d["x"], d["y"], 1.0, shadow=True)
    gate("c(p') euler", c.cpu().numpy(), r["c"], r["c_mag"])
    with pytest.raises(M.OcpError):
        H.vjp_params(x, wv)
    with H.params_bound(p2):
        with pytest.raises(M.OcpError):
            H.jprod(x, vn)
    H.close()


def test_bound_parameters_refuse_other_calls(M):
    """While the cart-pole's parameters are bound, the calls without a device-parameter variant
    (here eval_all) return OCP_EMODEL instead of silently using the host values."""
    w, d = case("cartpole_n1e5", 200)
    H = M.OCP.from_workload(w)
    x, y = dev(d["x"]), dev(d["y"])
    p = torch.tensor(w["params"], dtype=torch.float64, device="cuda")
    with H.params_bound(p):
        with pytest.raises(M.OcpError) as e:
            H.eval_all(x, y, 1.0)
        assert e.value.status == 5
    H.eval_all(x, y, 1.0)
    H.close()


@pytest.mark.parametrize("name,N", [("cartpole_n1e5", 6), ("goddard_n1e3", 5), ("quadrotor_n1e3", 4),
                                    ("vdp_n1e3", 9)])
def test_autograd_gradcheck_in_x_and_p(M, name, N):
    from paper_2510_03932_gb300 import autograd as A
    w, d = case(name, N)
    H = M.OCP.from_workload(w)
    x = dev(d["x"]).requires_grad_(True)
    p = torch.tensor(w["params"][:H.nparams], dtype=torch.float64, device="cuda", requires_grad=True)
    f = lambda x, p: A.constraints(H, x, p)
    assert torch.autograd.gradcheck(f, (x, p), eps=1e-6, atol=1e-6, rtol=1e-5)
    # second order in x (parameters held fixed)
    pc = p.detach()
    assert torch.autograd.gradgradcheck(lambda x: A.constraints(H, x, pc), (x,), eps=1e-6, atol=1e-5, rtol=1e-4)
    H.close()


def test_autograd_second_order_in_parameters_is_refused(M):
    from paper_2510_03932_gb300 import autograd as A
    w, d = case("cartpole_n1e5", 8)
    H = M.OCP.from_workload(w)
    x = dev(d["x"]).requires_grad_(True)
    p = torch.tensor(w["params"], dtype=torch.float64, device="cuda", requires_grad=True)
    gx, gp = torch.autograd.grad(A.constraints(H, x, p), (x, p), grad_outputs=dev(d["vm"]), create_graph=True)
    with pytest.raises(NotImplementedError):
        torch.autograd.grad(gp.sum(), (x,))
    H.close()


def test_autograd_parameter_gradient_against_oracle(M):
    """Cart-pole at N = 1e5: p.grad = (dc/dp)^T w and x.grad = J^T w against the oracle."""
    from paper_2510_03932_gb300 import autograd as A
    w = synth.workload("cartpole_n1e5")
    d = synth.draw(w)
    H = M.OCP.from_workload(w)
    P = O.Problem(w)
    x = dev(d["x"]).requires_grad_(True)
    p = torch.tensor(w["params"], dtype=torch.float64, device="cuda", requires_grad=True)
    (A.constraints(H, x, p) * dev(d["vm"])).sum().backward()
    ref, mag = O.dpar_vjp_all(P, d["x"], d["vm"], shadow=True)
    gate("p.grad", p.grad.cpu().numpy(), ref, mag)
    gx, gxm = O.jtprod(P, d["x"], d["vm"], shadow=True)
    gate("x.grad", x.grad.cpu().numpy(), gx, gxm)
    H.close()
