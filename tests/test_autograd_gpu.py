"""Differentiation form: torch.autograd Functions over the CUDA kernels.

Checked against central finite differences (torch.autograd.gradcheck / gradgradcheck in
FP64, eps = 1e-6) at small horizons, and against the CPU oracle's gradient (J^T w, the
mu-derivative and grad F) at the full N = 1e6 Van der Pol workload within the parity gate.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2510_03932_gb300 import synth
from parity import gate

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2510_03932_gb300 import autograd, ocp
    ocp.lib()
    return ocp, autograd


def small(name, N, **kw):
    w = dict(synth.with_horizon(synth.workload(name), N), **kw)
    d = synth.draw(w)
    return w, d


def test_constraints_gradcheck_vdp_mu(mods):
    ocp, A = mods
    w, d = small("vdp_n1e3", 12, params=[1.3])
    H = ocp.OCP.from_workload(w)
    x = torch.from_numpy(d["x"]).cuda().requires_grad_(True)
    mu = torch.tensor([1.3], dtype=torch.float64, device="cuda", requires_grad=True)
    f = lambda x, mu: A.constraints(H, x, mu)
    assert torch.autograd.gradcheck(f, (x, mu), eps=1e-6, atol=1e-7, rtol=1e-6)
    assert torch.autograd.gradgradcheck(f, (x, mu), eps=1e-6, atol=1e-6, rtol=1e-5)


def test_constraints_gradcheck_cartpole(mods):
    ocp, A = mods
    w, d = small("cartpole_n1e5", 6)
    H = ocp.OCP.from_workload(w)
    x = torch.from_numpy(d["x"]).cuda().requires_grad_(True)
    p = torch.tensor(w["params"], dtype=torch.float64, device="cuda")   # (m_c, m_p, l, g), held fixed
    f = lambda x: A.constraints(H, x, p)
    assert torch.autograd.gradcheck(f, (x,), eps=1e-6, atol=1e-6, rtol=1e-5)
    assert torch.autograd.gradgradcheck(f, (x,), eps=1e-6, atol=1e-5, rtol=1e-4)


@pytest.mark.parametrize("name,N", [("vdp_n1e3", 12), ("heat_n2e4", 3), ("quadrotor_n1e3", 4)])
def test_objective_gradcheck(mods, name, N):
    ocp, A = mods
    w, d = small(name, N)
    H = ocp.OCP.from_workload(w)
    x = torch.from_numpy(d["x"]).cuda().requires_grad_(True)
    f = lambda x: A.objective(H, x)
    assert torch.autograd.gradcheck(f, (x,), eps=1e-6, atol=1e-7, rtol=1e-6)
    assert torch.autograd.gradgradcheck(f, (x,), eps=1e-6, atol=1e-6, rtol=1e-5)


def test_backward_matches_oracle_at_full_size(mods):
    """Van der Pol with mu, N = 1e6: x.grad = J^T w, mu.grad = (dc/dmu)^T w, and the objective
    gradient, against the oracle within the parity gate."""
    ocp, A = mods
    w = dict(synth.workload("vdp_mu_n1e6"), params=[1.2])
    d = synth.draw(w)
    P = O.Problem(w, mu=1.2)
    H = ocp.OCP.from_workload(w)
    x = torch.from_numpy(d["x"]).cuda().requires_grad_(True)
    mu = torch.tensor([1.2], dtype=torch.float64, device="cuda", requires_grad=True)
    wv = torch.from_numpy(d["vm"]).cuda()
    c = A.constraints(H, x, mu)
    # forward value against the oracle
    ref = O.evaluate(P, d["x"], d["y"], 1.0, shadow=True)
    gate("c", c.detach().cpu().numpy(), ref["c"], ref["c_mag"])
    (c * wv).sum().backward()
    gx, gxm = O.jtprod(P, d["x"], d["vm"], shadow=True)
    gate("J^T w", x.grad.cpu().numpy(), gx, gxm)
    gmu, gmum = O.dpar_vjp(P, d["x"], d["vm"], shadow=True)
    gate("dc/dmu^T w", mu.grad.cpu().numpy(), np.array([gmu]), np.array([gmum]))
    x.grad = None
    F = A.objective(H, x)
    F.backward()
    gate("grad F", x.grad.cpu().numpy(), ref["g"], ref["g_mag"])
    gate("F", np.array([F.item()]), np.array([ref["f"]]), np.array([ref["f_mag"]]))


def test_param_binding_is_scoped(mods):
    """After an autograd call the handle reads mu from its host value again."""
    ocp, A = mods
    w, d = small("vdp_n1e3", 50, params=[1.0])
    H = ocp.OCP.from_workload(w)
    x = torch.from_numpy(d["x"]).cuda()
    c_host = H.eval_cons(x).clone()
    mu = torch.tensor([2.0], dtype=torch.float64, device="cuda")
    c_dev = A.constraints(H, x, mu)
    c_after = H.eval_cons(x)
    torch.cuda.synchronize()
    assert torch.equal(c_after, c_host)
    assert not torch.equal(c_dev, c_host)


def test_first_order_backward_equals_differentiable_backward(mods):
    """Without create_graph the backward is one direct launch (ocp_vjp_param_p); with it, the
    differentiable _ConsVJP Function.  Both run the same kernel: bit-identical results."""
    ocp, A = mods
    w, d = small("vdp_n1e3", 700, params=[0.8])
    H = ocp.OCP.from_workload(w)
    x = torch.from_numpy(d["x"]).cuda().requires_grad_(True)
    mu = torch.tensor([0.8], dtype=torch.float64, device="cuda", requires_grad=True)
    wv = torch.from_numpy(d["vm"]).cuda()
    g1 = torch.autograd.grad(A.constraints(H, x, mu), (x, mu), grad_outputs=wv)
    g2 = torch.autograd.grad(A.constraints(H, x, mu), (x, mu), grad_outputs=wv, create_graph=True)
    assert torch.equal(g1[0], g2[0].detach()) and torch.equal(g1[1], g2[1].detach())
    # mu read from the device tensor: a different mu changes both outputs
    mu2 = torch.tensor([1.1], dtype=torch.float64, device="cuda", requires_grad=True)
    g3 = torch.autograd.grad(A.constraints(H, x, mu2), (x, mu2), grad_outputs=wv)
    assert not torch.equal(g1[0], g3[0])
    H.close()


def test_whole_step_graph_replay_matches_eager(mods):
    """Forward and backward captured once in a CUDA graph over static x, mu, w; a replay after
    new values are copied into them equals the eager step bit for bit."""
    ocp, A = mods
    w, d = small("vdp_n1e3", 2000, params=[1.0])
    H = ocp.OCP.from_workload(w)
    xs = torch.from_numpy(d["x"]).cuda().requires_grad_(True)
    mus = torch.tensor([1.0], dtype=torch.float64, device="cuda", requires_grad=True)
    ws = torch.from_numpy(d["vm"]).cuda()

    def step():
        return torch.autograd.grad(A.constraints(H, xs, mus), (xs, mus), grad_outputs=ws)

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(3):
            step()
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        gx, gmu = step()
    d2 = synth.draw(w, seed=w["seed"] + 5)
    with torch.no_grad():
        xs.copy_(torch.from_numpy(d2["x"]))
        mus.fill_(0.7)
        ws.copy_(torch.from_numpy(d2["vm"]))
    g.replay()
    torch.cuda.synchronize()
    ex, emu = step()
    assert torch.equal(gx, ex) and torch.equal(gmu, emu)
    H.close()
