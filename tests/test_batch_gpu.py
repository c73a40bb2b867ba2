"""Batched form: many cart-pole (and Van der Pol) problems with uneven horizons in one
persistent launch.  Every instance slice must be bit-identical to the plain evaluator of
that instance (same per-node arithmetic), for every launch configuration; the objective of
each instance agrees within the parity gate; graph replay reproduces the direct launch; the
slices also agree with the CPU oracle."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2510_03932_gb300 import synth
from parity import gate

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ocp():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2510_03932_gb300 import ocp as M
    M.lib()
    return M


def make(ocp, ws):
    probs = [ocp.OCP.from_workload(w) for w in ws]
    B = ocp.OCPBatch(probs)
    draws = [synth.draw(w) for w in ws]
    x = torch.from_numpy(np.concatenate([d["x"] for d in draws])).cuda()
    y = torch.from_numpy(np.concatenate([d["y"] for d in draws])).cuda()
    return probs, B, draws, x, y


def batch_ws(model, Ns):
    ws = synth.batch_workloads(count=len(Ns), seed=77)
    if model == "vdp":
        base = synth.workload("vdp_n1e3")
        ws = [dict(base, N=int(N), seed=500 + i) for i, N in enumerate(Ns)]
    else:
        ws = [dict(w, N=int(N)) for w, N in zip(ws, Ns)]
    return ws


@pytest.mark.parametrize("model", ["cartpole", "vdp"])
def test_batch_slices_bit_identical_every_config(ocp, model):
    Ns = [1, 2, 63, 64, 127, 255, 256, 511, 1000, 2049]
    probs, B, draws, x, y = make(ocp, batch_ws(model, Ns))
    sigma = 0.8
    plain = []
    for P, d in zip(probs, draws):
        plain.append([t.cpu().numpy() for t in P.eval_all(torch.from_numpy(d["x"]).cuda(),
                                                          torch.from_numpy(d["y"]).cuda(), sigma)])
    for npt in (1, 2):
        for threads in (64, 128, 256):
            B.set_config(npt, threads, 0)
            f, c, g, jv, hv = B.outputs()
            for t in (f, c, g, jv, hv):
                t.fill_(float("nan"))
            B.eval_all(x, y, sigma, f, c, g, jv, hv)
            torch.cuda.synchronize()
            fh, ch, gh, jh, hh = (t.cpu().numpy() for t in (f, c, g, jv, hv))
            for i, (pf, pc, pg, pj, ph) in enumerate(plain):
                assert np.array_equal(ch[B.coff[i]:B.coff[i + 1]], pc), (npt, threads, i, "c")
                assert np.array_equal(gh[B.xoff[i]:B.xoff[i + 1]], pg), (npt, threads, i, "g")
                assert np.array_equal(jh[B.joff[i]:B.joff[i + 1]], pj), (npt, threads, i, "jac")
                assert np.array_equal(hh[B.hoff[i]:B.hoff[i + 1]], ph), (npt, threads, i, "hess")
                assert abs(fh[i] - pf[0]) <= 1e-12 * abs(pf[0]), (npt, threads, i, "f")


def test_batch_against_oracle_graph_and_autotune(ocp):
    Ns = [3, 700, 1500, 5001]
    ws = batch_ws("cartpole", Ns)
    probs, B, draws, x, y = make(ocp, ws)
    f, c, g, jv, hv = B.outputs()
    best = B.autotune(x, y, 1.0, f, c, g, jv, hv)
    assert best > 0
    cfg = B.get_config()
    assert cfg["threads"] in (64, 128, 256) and cfg["nodes_per_thread"] in (1, 2)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        B.eval_all(x, y, 1.0, f, c, g, jv, hv, stream=s)
    s.synchronize()
    ref = [t.clone() for t in (f, c, g, jv, hv)]
    for t in (f, c, g, jv, hv):
        t.zero_()
    torch.cuda.synchronize()
    B.graph_capture(x, y, 1.0, f, c, g, jv, hv, stream=s)
    B.graph_launch(stream=s)
    s.synchronize()
    for a, b in zip((f, c, g, jv, hv), ref):
        assert torch.equal(a, b)
    fh, ch, gh, jh, hh = (t.cpu().numpy() for t in (f, c, g, jv, hv))
    for i, (w, d) in enumerate(zip(ws, draws)):
        P = O.Problem(w)
        r = O.evaluate(P, d["x"], d["y"], 1.0, shadow=True)
        gate("f%d" % i, fh[i:i + 1], np.array([r["f"]]), np.array([r["f_mag"]]))
        gate("c%d" % i, ch[B.coff[i]:B.coff[i + 1]], r["c"], r["c_mag"])
        gate("g%d" % i, gh[B.xoff[i]:B.xoff[i + 1]], r["g"], r["g_mag"])
        gate("j%d" % i, jh[B.joff[i]:B.joff[i + 1]], r["jac"], r["jac_mag"])
        gate("h%d" % i, hh[B.hoff[i]:B.hoff[i + 1]], r["hess"], r["hess_mag"])


def test_batch_rejects_mixed_models(ocp):
    a = ocp.OCP.from_workload(synth.with_horizon(synth.workload("vdp_n1e3"), 10))
    b = ocp.OCP.from_workload(synth.with_horizon(synth.workload("cartpole_n1e5"), 10))
    with pytest.raises(ocp.OcpError):
        ocp.OCPBatch([a, b])
    h = ocp.OCP.from_workload(synth.with_horizon(synth.workload("heat_n2e4"), 10))
    with pytest.raises(ocp.OcpError):
        ocp.OCPBatch([h])
