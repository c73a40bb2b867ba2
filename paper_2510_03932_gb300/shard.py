"""One transcription split over S devices (contiguous node shards), one rank per device.

Shard s owns nodes [a_s, b_s) of 0..N and the defect rows j in [a_s, min(b_s, N)); it reads
x on nodes a_s..min(b_s, N) (a one-node halo on the right) and y on rows a_s-1..b_s-1 (the
multipliers of the row to its left).  Every output slot belongs to exactly one shard, so the
shards' outputs are concatenated without exchange; the objective and the parameter derivative
(dc/dmu)^T w are sums of the shard partials, added in rank order.  On the device a shard is one
ocp_eval_step_range (or ocp_eval_all_range, ocp_vjp_param_range) call; ShardedOCP runs a rank's
shard and combines the partials through torch.distributed.
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
    if nb > nx and a <= N < b:   # final rows X_{N,k} (every component or a subset)
        out["c"].append((nx, nb))
        out["jac"].append((nx, nb))
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


class ShardedOCP:
    """One problem evaluated by every rank of a torch.distributed process group, each rank on
    its own node shard and device.

    Every rank holds the inputs in the global layout (it reads only its shard and the one-node
    halo) and full-size output buffers of which it writes the slots `owned` lists.  The two
    cross-node sums are combined by gathering one double per rank (all_gather: device tensors
    with NCCL, host tensors with gloo) and adding the partials in rank order on the device
    (ocp_sum_ordered), so every rank ends with the same bits.  Nothing else moves between
    ranks.  The objective of the whole problem equals the unsharded one within rounding (the
    partials group the terms differently); every other output slot is bit-identical to the
    unsharded evaluation's.
    """

    def __init__(self, w: dict, group=None, rank: int | None = None, world: int | None = None):
        import torch.distributed as dist

        from . import ocp
        self.group = group
        self.rank = dist.get_rank(group) if rank is None else rank
        self.world = dist.get_world_size(group) if world is None else world
        self.H = ocp.OCP.from_workload(w)
        self.a, self.b = node_shards(self.H.N, self.world)[self.rank]
        self.layout = self.H.value_layout()
        self.owned = shard_slots(self.layout, self.a, self.b)

    def close(self):
        self.H.close()

    def combine(self, part, out=None, stream=None):
        """Sum over the ranks of the CUDA tensor `part` (k doubles), entry by entry in rank
        order, into `out`: one all-gather of k doubles per rank."""
        import torch
        import torch.distributed as dist

        from . import ocp
        out = part if out is None else out
        k = part.numel()
        if dist.get_backend(self.group) == "nccl":
            parts = torch.empty(self.world * k, dtype=torch.float64, device=part.device)
            dist.all_gather_into_tensor(parts, part.reshape(k), group=self.group)
        else:
            host = part.detach().reshape(k).cpu()
            gathered = [torch.empty_like(host) for _ in range(self.world)]
            dist.all_gather(gathered, host, group=self.group)
            parts = torch.cat(gathered).to(part.device)
        if k == 1:
            return ocp.sum_ordered(parts, out, stream)
        byentry = parts.reshape(self.world, k).t().contiguous()   # entry i's shares, rank order
        flat = out.reshape(k)
        for i in range(k):
            ocp.sum_ordered(byentry[i], flat[i:i + 1], stream)
        return out

    def eval_step(self, x, y, sigma, vn, vm, outs, stream=None):
        """This rank's shard of the fused step into the full-size buffers `outs` = (f, c, g,
        jvals, hvals, Jv, Jtv, Hv); f becomes the objective of the whole problem."""
        outs = self.H.eval_step_range(self.a, self.b, x, y, sigma, vn, vm, outs, stream)
        self.combine(outs[0], stream=stream)
        return outs

    def vjp_param(self, x, w, Jtw, dmu, stream=None):
        """This rank's entries of J^T w and the whole (dc/dmu)^T w (Van der Pol)."""
        self.H.vjp_param_range(self.a, self.b, x, w, Jtw, dmu, stream)
        self.combine(dmu, stream=stream)
        return Jtw, dmu

    def vjp_params(self, x, w, Jtw, dp, p=None, stream=None):
        """This rank's entries of J^T w and the whole (dc/dp)^T w for every dynamics parameter
        (p: device parameters, or None for the handle's)."""
        self.H.vjp_params_range(self.a, self.b, x, w, Jtw, dp, p, stream)
        self.combine(dp, stream=stream)
        return Jtw, dp

    # the product outputs share the slots of c (Jv) and g (J^T w, H v)
    _SLOTS = {"c": "c", "g": "g", "jac": "jac", "hess": "hess", "Jv": "c", "Jtv": "g", "Hv": "g"}

    def gather(self, name, t):
        """The complete output `name` (c, g, jac, hess, Jv, Jtv or Hv) on every rank, assembled
        from the ranks' owned slots (for checks; moves the whole array).  Path-inequality rows
        are not part of the slot bookkeeping."""
        import torch
        import torch.distributed as dist
        slots = self.owned[self._SLOTS[name]]
        host = t.detach().cpu()
        mine = torch.cat([host[s0:s1] for s0, s1 in slots]) if slots else host[:0]
        everyone = [None] * self.world
        dist.all_gather_object(everyone, (slots, mine), group=self.group)
        full = torch.full_like(host, float("nan"))
        for slots, vals in everyone:
            k = 0
            for s0, s1 in slots:
                full[s0:s1] = vals[k:k + s1 - s0]
                k += s1 - s0
        return full
