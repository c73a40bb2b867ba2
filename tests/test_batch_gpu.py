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
    if model in ("vdp", "dint", "quadrotor"):
        base = synth.workload({"vdp": "vdp_n1e3", "dint": "dint", "quadrotor": "quadrotor_n1e3"}[model])
        ws = [synth.with_horizon(dict(base, seed=500 + i), int(N)) for i, N in enumerate(Ns)]
    else:
        ws = [dict(w, N=int(N)) for w, N in zip(ws, Ns)]
    return ws


CONFIGS = [(npt, threads) for npt in (1, 2) for threads in (64, 128, 256)]


def provided(model, npt, threads):
    """The quadrotor's staged Jacobian rows (68 entries per node) fit 128 nodes per CTA."""
    return model != "quadrotor" or npt * threads <= 128


@pytest.mark.parametrize("model", ["cartpole", "vdp", "dint", "quadrotor"])
def test_batch_slices_bit_identical_every_config(ocp, model):
    Ns = [1, 2, 63, 64, 127, 255, 256, 511, 1000, 2049]
    probs, B, draws, x, y = make(ocp, batch_ws(model, Ns))
    sigma = 0.8
    plain = []
    for P, d in zip(probs, draws):
        plain.append([t.cpu().numpy() for t in P.eval_all(torch.from_numpy(d["x"]).cuda(),
                                                          torch.from_numpy(d["y"]).cuda(), sigma)])
    for npt, threads in CONFIGS:
        if not provided(model, npt, threads):
            with pytest.raises(ocp.OcpError) as e:
                B.set_config(npt, threads, 0)
            assert e.value.status == 1
            continue
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


def test_batch_quadrotor_autotune_skips_configs_it_cannot_fit(ocp):
    """The autotuner times only the configurations the quadrotor's shared memory allows and the
    tuned batch still equals the plain evaluator slice for slice."""
    ws = batch_ws("quadrotor", [1, 200, 1003, 64])
    probs, B, draws, x, y = make(ocp, ws)
    f, c, g, jv, hv = B.outputs()
    assert B.autotune(x, y, 1.0, f, c, g, jv, hv) > 0
    cfg = B.get_config()
    assert cfg["nodes_per_thread"] * cfg["threads"] <= 128
    B.eval_all(x, y, 1.0, f, c, g, jv, hv)
    torch.cuda.synchronize()
    for i, (P, d) in enumerate(zip(probs, draws)):
        pc, pj = (t.cpu().numpy() for t in P.eval_all(torch.from_numpy(d["x"]).cuda(),
                                                      torch.from_numpy(d["y"]).cuda(), 1.0)[2:4])
        assert np.array_equal(g[B.xoff[i]:B.xoff[i + 1]].cpu().numpy(), pc)
        assert np.array_equal(jv[B.joff[i]:B.joff[i + 1]].cpu().numpy(), pj)


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


def test_batch_full_workload_as_benchmarked(ocp):
    """The benchmark's batch (256 cart-pole instances, N ~ U{500..50000}, 6.5e6 nodes) in the
    benchmark's launch configuration (autotuned, replayed from a CUDA graph): eight instances
    (the shortest, the longest and six drawn at random) against the oracle through the parity
    gate and bit for bit against the plain evaluator."""
    ws = synth.batch_workloads()
    probs, B, draws, x, y = make(ocp, ws)
    f, c, g, jv, hv = B.outputs()
    B.autotune(x, y, 1.0, f, None, g, jv, hv)
    s = torch.cuda.Stream()
    for t in (f, g, jv, hv):
        t.fill_(float("nan"))
    torch.cuda.synchronize()
    B.graph_capture(x, y, 1.0, f, None, g, jv, hv, stream=s)
    B.graph_launch(stream=s)
    s.synchronize()
    Ns = np.array([w["N"] for w in ws])
    rng = np.random.default_rng(2026)
    pick = sorted({int(np.argmin(Ns)), int(np.argmax(Ns))} | set(rng.choice(len(ws), 6, replace=False).tolist()))
    fh, gh, jh, hh = (t.cpu().numpy() for t in (f, g, jv, hv))
    for i in pick:
        w, d = ws[i], draws[i]
        r = O.evaluate(O.Problem(w), d["x"], d["y"], 1.0, shadow=True)
        gate("f%d" % i, fh[i:i + 1], np.array([r["f"]]), np.array([r["f_mag"]]))
        gate("g%d" % i, gh[B.xoff[i]:B.xoff[i + 1]], r["g"], r["g_mag"])
        gate("j%d" % i, jh[B.joff[i]:B.joff[i + 1]], r["jac"], r["jac_mag"])
        gate("h%d" % i, hh[B.hoff[i]:B.hoff[i + 1]], r["hess"], r["hess_mag"])
        pf, pc, pg, pj, ph = (t.cpu().numpy() for t in probs[i].eval_all(torch.from_numpy(d["x"]).cuda(),
                                                                         torch.from_numpy(d["y"]).cuda(), 1.0))
        assert np.array_equal(gh[B.xoff[i]:B.xoff[i + 1]], pg)
        assert np.array_equal(jh[B.joff[i]:B.joff[i + 1]], pj)
        assert np.array_equal(hh[B.hoff[i]:B.hoff[i + 1]], ph)
    assert np.isfinite(gh).all() and np.isfinite(jh).all() and np.isfinite(hh).all() and np.isfinite(fh).all()


def test_batch_rejects_mixed_models(ocp):
    a = ocp.OCP.from_workload(synth.with_horizon(synth.workload("vdp_n1e3"), 10))
    b = ocp.OCP.from_workload(synth.with_horizon(synth.workload("cartpole_n1e5"), 10))
    with pytest.raises(ocp.OcpError):
        ocp.OCPBatch([a, b])
    h = ocp.OCP.from_workload(synth.with_horizon(synth.workload("heat_n2e4"), 10))
    with pytest.raises(ocp.OcpError):
        ocp.OCPBatch([h])


def test_autotune_cache_reuses_the_stored_configuration(tmp_path, monkeypatch):
    """With OCP_AUTOTUNE_CACHE set, the first autotune writes its result, keyed by the batch
    shape; a second batch of the same shape takes the stored configuration and time without
    timing, and a different shape is tuned again."""
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2510_03932_gb300 import ocp
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("OCP_AUTOTUNE_CACHE", str(path))

    def make(ns):
        ws = [synth.with_horizon(synth.workload("cartpole_n1e5"), n) for n in ns]
        probs = [ocp.OCP.from_workload(w) for w in ws]
        B = ocp.OCPBatch(probs)
        ds = [synth.draw(w) for w in ws]
        x = torch.from_numpy(np.concatenate([d["x"] for d in ds])).cuda()
        y = torch.from_numpy(np.concatenate([d["y"] for d in ds])).cuda()
        return probs, B, x, y

    probs, B, x, y = make([900, 2000, 4100])
    f, c, g, jv, hv = B.outputs()
    ms1 = B.autotune(x, y, 1.0, f, None, g, jv, hv)
    lines = path.read_text().splitlines()
    assert len(lines) == 1 and "model=2 count=3" in lines[0]
    cfg1 = B.get_config()
    probs2, B2, x2, y2 = make([900, 2000, 4100])
    f2, c2, g2, jv2, hv2 = B2.outputs()
    ms2 = B2.autotune(x2, y2, 1.0, f2, None, g2, jv2, hv2)
    assert B2.get_config() == cfg1 and abs(ms2 - ms1) <= 1e-6 * max(ms1, 1.0)
    assert len(path.read_text().splitlines()) == 1   # nothing re-timed
    B2.eval_all(x2, y2, 1.0, f2, None, g2, jv2, hv2)
    torch.cuda.synchronize()
    probs3, B3, x3, y3 = make([900, 2000])
    f3, c3, g3, jv3, hv3 = B3.outputs()
    B3.autotune(x3, y3, 1.0, f3, None, g3, jv3, hv3)
    assert len(path.read_text().splitlines()) == 2
    for P in probs + probs2 + probs3:
        P.close()
