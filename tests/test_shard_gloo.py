"""Multi-device sharding host logic, run as two gloo ranks on the CPU (no GPU).

Each rank takes its contiguous node shard, computes the output slots it owns and its
partial objective; the ranks exchange them (all_gather) and check that the slots of all
shards tile every output exactly once and that the rank-ordered sum of the partials equals
the oracle's objective of the whole problem.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import oracle as O
from paper_2510_03932_gb300 import shard, synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _partial_objective(w, x, a, b):
    """sum_{j in [a, b)} w_j f0(z_j) with the trapezoid weights of the whole horizon."""
    nx, nu, N, h = w["nx"], w["nu"], w["N"], w["T"] / w["N"]
    q, r = np.array(w["q"]), np.array(w["r"])
    X = x[: nx * (N + 1)].reshape(N + 1, nx)
    U = x[nx * (N + 1):].reshape(N + 1, nu)
    tot = 0.0
    for j in range(a, b):
        wj = h / 2 if j in (0, N) else h
        tot += wj * (np.sum(q * (X[j] - np.array(w["xref"])) ** 2) + np.sum(r * (U[j] - np.array(w["uref"])) ** 2))
    return tot


def _rank(rank, world, port, name, N, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = synth.with_horizon(synth.workload(name), N)
        P = O.Problem(w)
        jr, _ = O.jac_structure(P)
        nb = w["nx"] * (2 if w.get("xf") is not None else 1)
        rows = jr[nb:]
        jcount = [int(np.sum((rows >= nb + k * N) & (rows < nb + (k + 1) * N))) // N for k in range(w["nx"])]
        hr, hc = O.hess_structure(P)
        nX = w["nx"] * (N + 1)
        layout = dict(nx=w["nx"], nu=w["nu"], N=N, nb=nb, has_final=w.get("xf") is not None, jcount=jcount,
                      hx=int(np.sum(hr < nX)) // (N + 1), hu=int(np.sum(hr >= nX)) // (N + 1))
        a, b = shard.node_shards(N, world)[rank]
        slots = shard.shard_slots(layout, a, b)
        d = synth.draw(w)
        part = _partial_objective(w, d["x"], a, b)
        gathered = [None] * world
        dist.all_gather_object(gathered, (slots, part))
        if rank == 0:
            sizes = dict(c=P.m, g=P.n, jac=P.nnzj, hess=P.nnzh)
            for k, size in sizes.items():
                cover = np.zeros(size, np.int64)
                for sl, _ in gathered:
                    for s0, s1 in sl[k]:
                        cover[s0:s1] += 1
                assert np.all(cover == 1), (k, np.unique(cover))
            F = shard.combine_objective([p for _, p in gathered])
            ref = O.evaluate(P, d["x"], d["y"], 1.0)["f"]
            assert abs(F - ref) <= 1e-12 * abs(ref), (F, ref)
        dist.barrier()
        q.put((rank, "ok"))
    except Exception as e:  # report to the parent instead of hanging it
        q.put((rank, repr(e)))
        raise
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name,N", [("vdp_n1e3", 1000), ("dint", 57), ("heat_n2e4", 40)])
def test_two_rank_shards_tile_outputs_and_sum_objective(name, N):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, name, N, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    assert all(msg == "ok" for _, msg in res), res


def test_node_shards_cover_in_order():
    for N, S in [(1, 2), (10, 3), (1000, 8), (7, 8)]:
        sh = shard.node_shards(N, S)
        assert sh[0][0] == 0 and sh[-1][1] == N + 1
        assert all(sh[i][1] == sh[i + 1][0] for i in range(S - 1))
