"""Host logic for splitting one transcription over S devices (contiguous node shards).

Shard s owns nodes [a_s, b_s) of 0..N and the defect rows j in [a_s, min(b_s, N)); it reads
x on nodes a_s..min(b_s, N) (a one-node halo on the right) and y on rows a_s-1..b_s-1 (the
multipliers of the row to its left).  Every output slot belongs to exactly one shard, so the
shards' outputs are concatenated without exchange; the objective is the sum of the shard
partials, added in rank order.  On the device a shard is one ocp_eval_all_range call.
"""
from __future__ import annotations


def node_shards(N: int, S: int):
    """[a_s, b_s) for s < S: N+1 nodes split as evenly as possible, in order."""
    nodes = N + 1
    base, extra = divmod(nodes, S)
    out, a = [], 0
    for s in range(S):
        b = a + base + (1 if s < extra else 0)
        out.append((a, b))
        a = b
    return out


def shard_slots(layout: dict, a: int, b: int):
    """Output index ranges written by the shard owning nodes [a, b).

    layout: nx, nu, N, nb (boundary rows), has_final, jcount (entries per row of each
    component), hx, hu (Hessian entries per node in the X and U blocks).
    Returns {output: [(start, stop), ...]} for c, g, jac, hess.
    """
    nx, nu, N, nb = layout["nx"], layout["nu"], layout["N"], layout["nb"]
    r0, r1 = a, min(b, N)
    out = {"c": [], "g": [], "jac": [], "hess": []}
    if a == 0:
        out["c"].append((0, nx))
        out["jac"].append((0, nx))
    if layout["has_final"] and a <= N < b:
        out["c"].append((nx, 2 * nx))
        out["jac"].append((nx, 2 * nx))
    base = nb
    for k in range(nx):
        cnt = layout["jcount"][k]
        if r1 > r0:
            out["c"].append((nb + k * N + r0, nb + k * N + r1))
            out["jac"].append((base + r0 * cnt, base + r1 * cnt))
        base += cnt * N
    out["g"].append((nx * a, nx * b))
    out["g"].append((nx * (N + 1) + nu * a, nx * (N + 1) + nu * b))
    hx, hu = layout["hx"], layout["hu"]
    if hx:
        out["hess"].append((hx * a, hx * b))
    if hu:
        out["hess"].append((hx * (N + 1) + hu * a, hx * (N + 1) + hu * b))
    return out


def combine_objective(partials):
    """Objective of the whole problem from the shard partials, added in rank order."""
    total = 0.0
    for p in partials:
        total += float(p)
    return total
