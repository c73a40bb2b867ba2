"""The sharded evaluator with real shards: two or three processes share the GPU, each runs its
own node shard through ocp_eval_step_range / ocp_vjp_param_range / ocp_vjp_params_range
(ShardedOCP), and the ranks combine their partials over gloo.  The assembled outputs must equal
the unsharded fused step bit for bit, and the combined objective, (dc/dmu)^T w and (dc/dp)^T w
for every dynamics parameter must agree with the oracle within the parity gate.  (The ranks never wait on each other inside a kernel: every exchange happens on
the host, between launches.)"""
import os
import socket
import sys

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, name, N, q):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as O
        from paper_2510_03932_gb300 import ocp, synth
        from paper_2510_03932_gb300.shard import ShardedOCP
        from parity import gate
        from test_parity_gpu import named

        torch.cuda.set_device(0)
        w = named(name, N)
        d = synth.draw(w)
        S = ShardedOCP(w)
        x, y, vn, vm = (torch.from_numpy(d[k]).cuda() for k in ("x", "y", "vn", "vm"))
        H = S.H
        outs = tuple(torch.full((k,), float("nan"), dtype=torch.float64, device="cuda")
                     for k in (1, H.m, H.n, H.nnzj, H.nnzh, H.m, H.n, H.n))
        S.eval_step(x, y, w["sigma"], vn, vm, outs)
        names = ("c", "g", "jac", "hess", "Jv", "Jtv", "Hv")
        full = {nm: S.gather(nm, t) for nm, t in zip(names, outs[1:])}
        vjp = None
        if w["model"] == "vdp":
            Jtw = torch.full((H.n,), float("nan"), dtype=torch.float64, device="cuda")
            dmu = torch.zeros(1, dtype=torch.float64, device="cuda")
            S.vjp_param(x, vm, Jtw, dmu)
            vjp = (S.gather("Jtv", Jtw), float(dmu))
        vjps = None
        if H.nparams > 0:   # every dynamics parameter, read from a device tensor
            p = torch.tensor(w["params"][:H.nparams], dtype=torch.float64, device="cuda")
            Jtw = torch.full((H.n,), float("nan"), dtype=torch.float64, device="cuda")
            dp = torch.zeros(H.nparams, dtype=torch.float64, device="cuda")
            S.vjp_params(x, vm, Jtw, dp, p)
            vjps = (S.gather("Jtv", Jtw), dp.cpu().numpy())
            dps = [None] * world
            dist.all_gather_object(dps, vjps[1].tolist())
            assert all(v == dps[0] for v in dps), dps   # the same bits on every rank
        f = float(outs[0])
        fs = [None] * world
        dist.all_gather_object(fs, f)
        assert all(v == f for v in fs), fs   # every rank holds the same combined objective
        if rank == 0:
            # the unsharded fused step on the same inputs
            ref = H.eval_step(x, y, w["sigma"], vn, vm)
            for nm, t in zip(names, ref[1:]):
                assert torch.equal(full[nm], t.cpu()), nm
            P = O.Problem(w)
            ev = O.evaluate(P, d["x"], d["y"], w["sigma"], shadow=True)
            gate("f", np.array([f]), np.array([ev["f"]]), np.array([ev["f_mag"]]))
            if vjp is not None:
                Jtw_ref, dmu_ref = H.vjp_param(x, vm)
                assert torch.equal(vjp[0], Jtw_ref.cpu())
                o, m = O.dpar_vjp(P, d["x"], d["vm"], shadow=True)
                gate("dmu", np.array([vjp[1]]), np.array([o]), np.array([m]))
            if vjps is not None:
                Jtw_ref, _ = H.vjp_params(x, vm)
                assert torch.equal(vjps[0], Jtw_ref.cpu())
                o, m = O.dpar_vjp_all(P, d["x"], d["vm"], shadow=True)
                gate("dc/dp^T w", vjps[1], o, m)
        dist.barrier()
        S.close()
        q.put((rank, "ok"))
    except Exception as e:  # report to the parent instead of hanging it
        import traceback
        q.put((rank, repr(e) + traceback.format_exc()[-1500:]))
        raise
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name,N,world", [("vdp_mu_n1e6", 100000, 2), ("vdp_n1e3", 1000, 3),
                                          ("cartpole_n1e5", 20000, 2), ("quadrotor_n1e3", 5000, 3),
                                          ("dint", 300, 2)])
def test_sharded_step_equals_unsharded(name, N, world):
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, name, N, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    assert all(msg == "ok" for _, msg in res), res
