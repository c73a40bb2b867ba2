"""Benchmark: Jacobian + Hessian COO nonzeros per second (FP64) of the trapezoidal
transcription evaluator on GB300, with the HBM roofline fraction of the dominant kernel.

One step = one pass of the hot path on one problem (ocp_eval_step, one launch): objective,
constraints, gradient, Jacobian and Hessian values and the three products Jv, J^T v and H v.  value = (nnz_J + nnz_H) * steps * ranks / (max over ranks of the summed
step times).  Inputs are resident in HBM; between timed steps the L2 is flushed by
writing a 512 MB buffer and reading it back (outside the timed events; L2Flush).  `e2e` repeats the step through the
host-buffer call ocp_eval_step_host_async (pinned host arrays in and out, every host<->device
copy inside the timed region, joined by ocp_host_step_wait before the end event).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Under torchrun (N > 1) every rank evaluates its own instance (weak scaling, no collective
in the data path); rank 0 prints the JSON line.
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2510_03932_gb300 import synth  # noqa: E402

METRIC = "Jac+Hess COO nnz/s (FP64) and % HBM roofline; batched/adjoint vs plain, 1e-12"
DEFAULT_WORKLOAD = "vdp_mu_n1e6"


def tracked_components(w):
    """State components with a time-varying reference (their per-node table is read too)."""
    sl, am, fr = (w.get(k) or [0.0] * w["nx"] for k in ("xslope", "xamp", "xfreq"))
    return sum(1 for k in range(w["nx"]) if sl[k] != 0.0 or (am[k] != 0.0 and fr[k] != 0.0))


def algorithmic_bytes(w, kind):
    """Bytes each kernel must move at least once: inputs read once, outputs written once."""
    n, m = synth.dims(w)
    P = _counts(w)
    nnzj, nnzh = P
    trk = tracked_components(w) * (w["N"] + 1)   # reference table, read by F and grad
    if kind == "eval_all":
        return 8 * (n + m + 1 + m + n + nnzj + nnzh + trk)
    if kind == "step":  # reads x, y, vn, vm; writes f, c, g, J, H, Jv, J^T w, Hv
        return 8 * (n + m + n + m + 1 + m + n + nnzj + nnzh + m + n + n + trk)
    if kind == "jh":
        return 8 * (n + m + nnzj + nnzh)
    if kind == "jprod":
        return 8 * (n + n + m)
    if kind == "jtprod":
        return 8 * (n + m + n)
    if kind == "hprod":
        return 8 * (n + m + n + n)
    raise KeyError(kind)


_COUNT_CACHE = {}


def _counts(w):
    key = (ops_model(w), w["nx"], w["N"], tuple(w["q"]), tuple(w["r"]), w.get("xf") is not None,
           w.get("scheme", "trapezoid"), bool(w.get("free_tf")), tuple(w.get("xf_comp") or ()))
    if key not in _COUNT_CACHE:
        from paper_2510_03932_gb300 import ocp
        H = ocp.OCP.from_workload(w)
        _COUNT_CACHE[key] = (H.nnzj, H.nnzh)
        H.close()
    return _COUNT_CACHE[key]


# FP64 arithmetic instructions (DFMA + DADD + DMUL per thread) each kernel executes per node:
# ncu's sm__sass_thread_inst_executed_op_{dfma,dadd,dmul}_pred_on counts divided by N+1 (the
# objective's tile reduction is part of them).  The cart-pole's include a sincos and a division, the quadrotor's three sincos calls and
# 1/cos x8, the Goddard's exp and two divisions.  Measured at N = 1e5 (cart-pole, quadrotor,
# Goddard) and 1e6 (Van der Pol).  Each model's counts hold for the kernel sources whose tag
# (kernel_source_tag) is in FP64_OPS_SRC; when the sources change the counts are stale and the
# bench reports no FP64 fraction for that model until they are measured again.
FP64_OPS_PER_NODE = {("vdp", "eval_all"): 26.6, ("vdp", "jh"): 10.0, ("vdp", "jprod"): 13.0,
                     ("vdp", "jtprod"): 12.0, ("vdp", "hprod"): 11.0, ("vdp", "step"): 50.6,
                     ("cartpole", "eval_all"): 109.7, ("cartpole", "jh"): 87.7, ("cartpole", "jprod"): 74.6,
                     ("cartpole", "jtprod"): 71.0, ("cartpole", "hprod"): 89.0, ("cartpole", "step"): 156.9,
                     ("quadrotor", "eval_all"): 235.5, ("quadrotor", "jh"): 163.3, ("quadrotor", "jprod"): 151.2,
                     ("quadrotor", "jtprod"): 143.0, ("quadrotor", "hprod"): 186.0, ("quadrotor", "step"): 382.8,
                     ("goddard", "eval_all"): 94.2, ("goddard", "jh"): 85.2, ("goddard", "jprod"): 62.3,
                     ("goddard", "jtprod"): 62.1, ("goddard", "hprod"): 89.1, ("goddard", "step"): 149.3,
                     ("vdp:euler", "eval_all"): 21.5, ("vdp:euler", "jh"): 8.0, ("vdp:euler", "jprod"): 11.0,
                     ("vdp:euler", "jtprod"): 10.0, ("vdp:euler", "hprod"): 10.0, ("vdp:euler", "step"): 41.5,
                     # heat, 64 cells: the step is its evaluation and one launch of Jv, J^T w and H v
                     ("heat64", "eval_all"): 1122.8, ("heat64", "jh"): 390.4, ("heat64", "jprod"): 523.4,
                     ("heat64", "jtprod"): 463.0, ("heat64", "hprod"): 257.0, ("heat64", "step"): 2366.2}

# The kernel sources of each model key (paths under the package's csrc/): the tile body and
# the helpers it includes, the model's device functor, the translation unit that instantiates
# its kernels.
_COMMON = ["node_kernels.cuh", "model_base.cuh", "kernel_config.h"]
KERNEL_SOURCES = {
    "vdp": _COMMON + ["model_vdp.cuh", "node_vdp.cu"],
    "vdp:euler": _COMMON + ["model_vdp.cuh", "node_vdp.cu"],
    "cartpole": _COMMON + ["model_cartpole.cuh", "node_cartpole.cu", "sincos_table.cuh", "sincos_table_data.h"],
    "quadrotor": _COMMON + ["model_quad.cuh", "node_quad.cu", "sincos_table.cuh", "sincos_table_data.h"],
    "goddard": _COMMON + ["goddard_kernels.cu", "exp_table.cuh", "exp_table_data.h"],
    "heat64": _COMMON + ["heat_kernels.cu"],
}
# Tags of the sources the FP64_OPS_PER_NODE counts (and TRAFFIC) were measured on.
FP64_OPS_SRC = {"vdp": "76d84f0080b4", "vdp:euler": "76d84f0080b4", "cartpole": "810d82f3b0b7",
                "quadrotor": "d9efc5bf84c0", "goddard": "5f8786230bfe", "heat64": "6e2d20e68d84"}


def kernel_source_tag(key):
    """First 12 hex digits of the SHA-256 of the model's kernel sources (KERNEL_SOURCES)."""
    import hashlib
    hsh = hashlib.sha256()
    for rel in KERNEL_SOURCES[key]:
        with open(os.path.join(ROOT, "paper_2510_03932_gb300", "csrc", rel), "rb") as fh:
            hsh.update(rel.encode() + b"\0" + fh.read() + b"\0")
    return hsh.hexdigest()[:12]


def fp64_ops(key, kern):
    """The measured FP64 instructions per node of this kernel, or None when the model's
    kernel sources changed since the measurement (or it was never measured)."""
    if key not in FP64_OPS_SRC or kernel_source_tag(key) != FP64_OPS_SRC[key]:
        return None
    return FP64_OPS_PER_NODE.get((key, kern))


# Rows of the paper's workloads beyond the headline problem (and the cart-pole at the
# headline horizon), measured the same way (fused step with an L2 flush between steps) and
# reported under "widened".
WIDENED = ["cartpole_n1e6", "quadrotor_n1e6", "goddard_n1e6", "vdp_mu_n1e6:euler"]
# The paper's three plain evaluation workloads (Van der Pol N = 1e3, cart-pole N = 1e5, heat
# N = 2e4), timed the same way and reported under "configs".
CONFIGS = ["vdp_n1e3", "cartpole_n1e5", "heat_n2e4"]


def ops_model(w):
    """Key of FP64_OPS_PER_NODE: the model (heat with its cell count), with the scheme when it
    is not the trapezoid."""
    m = w["model"] + ("%d" % w["nx"] if w["model"] == "heat" else "")
    return m + (":euler" if w.get("scheme") == "euler" else "")


def named_workload(name):
    """A workload by name; the suffix ":euler" selects the forward Euler scheme."""
    base, _, scheme = name.partition(":")
    w = synth.workload(base)
    if scheme:
        w = dict(w, scheme=scheme, name=name)
    return w


# DRAM bytes (read + write) of one launch at a workload, from an ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum; writes still dirty in L2 when the kernel ends
# are not counted), with the source tag of the kernel it was captured on (see traffic()).
TRAFFIC = {("vdp_mu_n1e6", "step"): (227.69e6, "76d84f0080b4")}
# Each SM's FP64 pipe completes 2 FP64 instructions (one lane each) per clock: the recipe's
# nominal 1.25 TFLOP/s FP64 of GB300 is 6.25e11 FMA/s = 1.99 per clock per SM at 152 SMs and
# 2070 MHz.  bench.py measures the rate live (measure_fp64_rate) and reports it beside the peak.
FP64_INST_PER_CLK_PER_SM = 2.0
NUM_SMS = 152


def traffic(name, kern, key):
    """Measured DRAM bytes of one launch, or None once the kernel's sources have changed."""
    v = TRAFFIC.get((name, kern))
    if v is None or kernel_source_tag(key) != v[1]:
        return None
    return v[0]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class L2Flush:
    """Between timed calls: write a 512 MB buffer (four times the 129 MB L2), then read it back
    (a sum into one float), so that the next call finds none of its data in the L2 and no dirty
    line of the flush left to write back to DRAM while it runs (a write alone leaves up to the
    L2's size of dirty lines, whose write-back the next timed call would pay for)."""

    def __init__(self, dev):
        import torch
        self.buf = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        self.acc = torch.empty((), dtype=torch.float32, device=dev)

    def __call__(self):
        import torch
        self.buf.zero_()
        torch.sum(self.buf, dim=0, out=self.acc)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [s.strip() for s in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1])); mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def bench_config(name, w, n, m, nnzj, nnzh, world):
    """The `config` object of the JSON line (the same keys for both arms)."""
    return dict(workload=name, model=w["model"], N=w["N"], n=n, m=m, nnz_jac=nnzj, nnz_hess=nnzh,
                step="one pass of the hot path: F, c, grad, J, H, Jv, J^T w, Hv",
                l2="inputs and outputs (296 MB at the default workload) exceed the L2; between steps a 512 MB "
                   "write and read-back leave it cold and clean (no dirty line of the flush to write back)",
                parallelism="replicas" if world > 1 else "single")


def measure_fp64_rate(dev, nsm, seconds=0.25):
    """FP64 instructions per clock per SM of DFMA (register operands; multiplier from the
    constant bank), DADD and DMUL, from the library's throughput probe (ocp_probe_fp64): 8 CTAs
    of 256 threads per SM, each launch about `seconds` long, timed with CUDA events on the
    launching stream, with the SM clock sampled meanwhile."""
    import torch
    from paper_2510_03932_gb300 import ocp

    blocks, threads = 8 * nsm, 256
    out = torch.zeros(blocks * threads, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    ocp.probe_fp64(0, blocks, threads, 256, out, stream)   # warm-up
    torch.cuda.synchronize(dev)
    # size the launches from a short one: about `seconds` each at the rate it shows
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    nops = ocp.probe_fp64(0, blocks, threads, 4096, out, stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    rate = nops / (e0.elapsed_time(e1) * 1e-3)
    iters = int(max(1024, min(1 << 24, rate * seconds / (blocks * threads * 8))))
    sampler = ClockSampler(dev.index)
    sampler.start()
    res = {}
    for op, name in ((0, "dfma"), (1, "dadd"), (2, "dmul"), (3, "dfma_const_multiplier"), (4, "dfma_const_addend")):
        ms = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            nops = ocp.probe_fp64(op, blocks, threads, iters, out, stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms.append(e0.elapsed_time(e1))
        res[name] = nops / (float(np.median(ms)) * 1e-3)
    clocks = sampler.stop()
    clk = clocks.get("sm_mhz") or 2070.0
    per = {k: v / (clk * 1e6 * nsm) for k, v in res.items()}
    return dict(kernel="ocp_probe_fp64 (8 independent chains per thread, %d x %d threads, %d iterations)"
                       % (blocks, threads, iters),
                dfma_per_clk_per_sm=per["dfma"], dadd_per_clk_per_sm=per["dadd"], dmul_per_clk_per_sm=per["dmul"],
                dfma_const_multiplier_per_clk_per_sm=per["dfma_const_multiplier"],
                dfma_const_addend_per_clk_per_sm=per["dfma_const_addend"],
                dfma_G_per_s=res["dfma"] / 1e9, sm_mhz=clk, clocks=clocks)


def run_ours(args, rank, world):
    import torch
    from paper_2510_03932_gb300 import ocp

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    w = named_workload(args.workload)
    d = synth.draw(w, seed=w["seed"] + rank)
    H = ocp.OCP.from_workload(w)
    n, m, nnzj, nnzh = H.n, H.m, H.nnzj, H.nnzh
    sigma = w["sigma"]
    x = torch.from_numpy(d["x"]).to(dev)
    y = torch.from_numpy(d["y"]).to(dev)
    vn = torch.from_numpy(d["vn"]).to(dev)
    vm = torch.from_numpy(d["vm"]).to(dev)
    f = torch.empty(1, dtype=torch.float64, device=dev)
    c = torch.empty(m, dtype=torch.float64, device=dev)
    g = torch.empty(n, dtype=torch.float64, device=dev)
    jv = torch.empty(nnzj, dtype=torch.float64, device=dev)
    hv = torch.empty(nnzh, dtype=torch.float64, device=dev)
    Jv = torch.empty(m, dtype=torch.float64, device=dev)
    Jtv = torch.empty(n, dtype=torch.float64, device=dev)
    Hv = torch.empty(n, dtype=torch.float64, device=dev)
    flush = L2Flush(dev)
    stream = torch.cuda.current_stream(dev)
    names = ["eval_all", "jprod", "jtprod", "hprod"]
    outs = (f, c, g, jv, hv, Jv, Jtv, Hv)

    def step():
        # one pass of the hot path: F, c, grad, J, H and Jv, J^T w, Hv at the same x
        H.eval_step(x, y, sigma, vn, vm, outs)

    def separate(ev):
        ev[0].record(stream)
        H.eval_all(x, y, sigma, f, c, g, jv, hv, alloc=False)
        ev[1].record(stream)
        H.jprod(x, vn, Jv)
        ev[2].record(stream)
        H.jtprod(x, vm, Jtv)
        ev[3].record(stream)
        H.hprod(x, y, sigma, vn, Hv)
        ev[4].record(stream)

    for _ in range(args.warmup):
        flush()
        step()
    torch.cuda.synchronize(dev)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    sampler = ClockSampler(dev.index if rank == 0 else -1) if rank == 0 else None
    if sampler:
        sampler.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for k in range(args.steps):
        flush()
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop() if sampler else None
    step_ms = np.array([evs[k][0].elapsed_time(evs[k][1]) for k in range(args.steps)])
    tot_ms = float(step_ms.sum())
    if world > 1:
        t = torch.tensor([tot_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        tot_ms = float(t.item())
    # --- the same work as four separate calls (per-kernel breakdown)
    sev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(min(args.steps, 50))]
    for ev in sev:
        flush()
        separate(ev)
    torch.cuda.synchronize(dev)
    per = np.array([[ev[i].elapsed_time(ev[i + 1]) for i in range(4)] for ev in sev])
    kern_ms = per.mean(axis=0)
    # --- J+H alone (the fused Jacobian+Hessian values launch), timed the same way
    jh = []
    for k in range(min(args.steps, 50)):
        flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        H.eval_all(x, y, sigma, None, None, None, jv, hv, alloc=False)
        e1.record(stream)
        jh.append((e0, e1))
    torch.cuda.synchronize(dev)
    jh_ms = float(np.mean([a.elapsed_time(b) for a, b in jh]))
    # --- the same step replayed from a CUDA graph (flushed), and hot (no flush, labelled)
    graph_ms = None
    try:
        gs = torch.cuda.Stream(dev)
        gs.wait_stream(stream)
        with torch.cuda.stream(gs):
            for _ in range(2):
                step()
        stream.wait_stream(gs)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        gt = []
        for k in range(min(args.steps, 50)):
            flush()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            graph.replay()
            e1.record(stream)
            gt.append((e0, e1))
        torch.cuda.synchronize(dev)
        graph_ms = float(np.mean([a.elapsed_time(b) for a, b in gt]))
    except Exception:
        graph_ms = None
    ht = []
    for k in range(min(args.steps, 50)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        ht.append((e0, e1))
    torch.cuda.synchronize(dev)
    hot_ms = float(np.mean([a.elapsed_time(b) for a, b in ht[3:]]))
    # --- KKT assembly from the step's H and J values (HBM-bound gather), timed the same way
    sig_x = torch.ones(n, dtype=torch.float64, device=dev)
    kv = H.kkt_values(hv, jv, sig_x, 1e-8, 1e-8)
    kk = []
    for k in range(min(args.steps, 50)):
        flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        H.kkt_values(hv, jv, sig_x, 1e-8, 1e-8, out=kv)
        e1.record(stream)
        kk.append((e0, e1))
    torch.cuda.synchronize(dev)
    kkt_ms = float(np.mean([a.elapsed_time(b) for a, b in kk]))
    kkt_bytes = 8 * (nnzj + nnzh + n + kv.numel())
    # --- end to end: pinned host buffers, copies inside the timed region.  The step goes through
    # ocp_eval_step_host_async (host arrays in and out, copied whole on the library's copy
    # streams; the next step overlaps the previous step's output copy) with one
    # ocp_host_step_wait before the end event; the joined ocp_eval_step_host and the same copies
    # issued around the device step are timed beside it.
    hx = torch.from_numpy(d["x"]).pin_memory(); hy = torch.from_numpy(d["y"]).pin_memory()
    hvn = torch.from_numpy(d["vn"]).pin_memory(); hvm = torch.from_numpy(d["vm"]).pin_memory()
    outs = [f, c, g, jv, hv, Jv, Jtv, Hv]
    houts = tuple(torch.empty(t.numel(), dtype=torch.float64).pin_memory() for t in outs)
    e2e_steps = max(3, min(args.steps, 20))

    def host_step():
        H.eval_step_host(hx, hy, sigma, hvn, hvm, houts, stream)

    def host_step_async():
        H.eval_step_host(hx, hy, sigma, hvn, hvm, houts, stream, wait=False)

    def copy_then_step():
        x.copy_(hx, non_blocking=True); y.copy_(hy, non_blocking=True)
        vn.copy_(hvn, non_blocking=True); vm.copy_(hvm, non_blocking=True)
        step()
        for ho, t in zip(houts, outs):
            ho.copy_(t, non_blocking=True)

    def time_e2e(fn):
        ms = []
        for k in range(e2e_steps + 2):
            flush()
            # the host step's input copy does not wait for earlier work on the stream: the
            # flush must be over before the start event
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            if k >= 2:
                ms.append(e0.elapsed_time(e1))
        return ms

    def time_e2e_stream(fn, k):
        # k steps back to back on one stream (each with its own copies in and out; the inputs
        # and outputs, 296 MB a step at the default workload, exceed the L2): consecutive
        # calls overlap one step's input copy with the previous step's output copy; every
        # output copy is joined to the stream before the end event
        for _ in range(2):
            fn()
        H.host_step_wait(stream)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        H.host_step_wait(stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / k

    e2e_sync_ms = float(np.mean(time_e2e(host_step)))
    e2e_whole_ms = float(np.mean(time_e2e(copy_then_step)))
    e2e_joined_ms = time_e2e_stream(host_step, e2e_steps)
    e2e_ms = [time_e2e_stream(host_step_async, e2e_steps)]
    nnz = nnzj + nnzh
    e2e_val = nnz * world / (float(np.mean(e2e_ms)) * 1e-3)
    hbm, peak_kind = peaks()
    step_mean = tot_ms / args.steps
    ab = algorithmic_bytes(w, "step")
    achieved = ab / (step_mean * 1e-3) / 1e9
    clk = (clocks or {}).get("sm_mhz") or 2070.0
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp64_peak = FP64_INST_PER_CLK_PER_SM * nsm * clk * 1e6 / 1e9   # G FP64 inst/s
    key = ops_model(w)
    ops = fp64_ops(key, "step")
    fp64_ach = ops * (w["N"] + 1) / (step_mean * 1e-3) / 1e9 if ops else None
    probe = measure_fp64_rate(dev, nsm)
    jh_bytes = algorithmic_bytes(w, "jh")
    jh_gbps = jh_bytes / (jh_ms * 1e-3) / 1e9
    res = dict(
        metric=METRIC, value=nnz * args.steps * world / (tot_ms * 1e-3), unit="nnz/s", n_gpus=world,
        steps=args.steps, warmup=args.warmup, ms_per_step=tot_ms / args.steps, higher_is_better=True,
        scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
        config=bench_config(args.workload, w, n, m, nnzj, nnzh, world),
        roofline=dict(bound="alu", achieved=fp64_ach, peak=fp64_peak, unit="G FP64 inst/s",
                      frac=(fp64_ach / fp64_peak) if fp64_ach else None,
                      traffic=traffic(w["name"], "step", key),
                      kernel="k_node_eval<step> (fused step: F, c, grad, J, H, Jv, J^T w, Hv)",
                      fp64_inst_per_node=ops, fp64_counts_source_tag=kernel_source_tag(key),
                      fp64_counts_current=ops is not None,
                      peak_basis="%.0f FP64 inst/clk/SM (GB300's nominal 1.25 TFLOP/s FP64) x %d SMs x %.0f MHz "
                                 "(median SM clock under load)" % (FP64_INST_PER_CLK_PER_SM, nsm, clk),
                      peak_probe=probe,
                      # the Jacobian + Hessian values alone (one launch), against the HBM roofline
                      jac_hess=dict(bound="hbm", ms=jh_ms, nnz_per_s=nnz / (jh_ms * 1e-3), achieved=jh_gbps,
                                    peak=hbm, unit="GB/s", frac=jh_gbps / hbm, algorithmic_bytes=jh_bytes,
                                    peak_source=peak_kind, l2="flushed between calls (512 MB write, then read back)")),
        roofline_hbm=dict(bound="hbm", achieved=achieved, peak=hbm, unit="GB/s", frac=achieved / hbm,
                          peak_source=peak_kind, algorithmic_bytes=ab,
                          traffic=traffic(w["name"], "step", key)),
        separate_calls_ms=float(kern_ms.sum()),
        kernels={nm: dict(ms=float(kern_ms[i]), GBps=algorithmic_bytes(w, nm) / (kern_ms[i] * 1e-3) / 1e9,
                          hbm_frac=algorithmic_bytes(w, nm) / (kern_ms[i] * 1e-3) / 1e9 / hbm,
                          fp64_frac=(fp64_ops(key, nm) * (w["N"] + 1) / (kern_ms[i] * 1e-3) / 1e9
                                     / fp64_peak) if fp64_ops(key, nm) else None)
                 for i, nm in enumerate(names)},
        jac_hess_only=dict(ms=jh_ms, nnz_per_s=nnz / (jh_ms * 1e-3),
                           GBps=algorithmic_bytes(w, "jh") / (jh_ms * 1e-3) / 1e9,
                           frac=algorithmic_bytes(w, "jh") / (jh_ms * 1e-3) / 1e9 / hbm),
        step_graph_replay_ms=graph_ms,
        step_hot_ms=hot_ms,   # no L2 flush between steps (the 296 MB step does not fit L2)
        kkt_assembly=dict(ms=kkt_ms, nnz=kv.numel(), GBps=kkt_bytes / (kkt_ms * 1e-3) / 1e9,
                          hbm_frac=kkt_bytes / (kkt_ms * 1e-3) / 1e9 / hbm,
                          what="K = [H + diag(sigma_x + delta_w), J^T; J, -delta_c I] from the COO values"),
        e2e=dict(value=e2e_val, unit="nnz/s", h2d_bytes_per_step=8 * (n + m + n + m),
                 d2h_bytes_per_step=8 * sum(t.numel() for t in outs), ms=float(np.mean(e2e_ms)),
                 call="ocp_eval_step_host_async, %d steps back to back on one stream, then "
                      "ocp_host_step_wait" % e2e_steps,
                 joined_calls_ms=e2e_joined_ms,
                 synchronized_step_ms=e2e_sync_ms, whole_copies_around_device_step_ms=e2e_whole_ms),
        gpu_launches=args.steps, clocks=clocks, wall_s=wall,
    )
    return res


def run_sharded(args, rank, world):
    """One problem split over the ranks (ShardedOCP): every rank evaluates its own contiguous
    node shard of the workload on its own GPU (ocp_eval_step_range) and the partial objectives
    are combined in rank order (all_gather of one double per rank, ocp_sum_ordered).  value =
    the whole problem's nnz_J + nnz_H per step / the max over ranks of the step time (strong
    scaling).  e2e: each step also copies the rank's inputs in from pinned host memory and its
    owned output slots (and f) back."""
    import torch
    import torch.distributed as dist
    from paper_2510_03932_gb300.shard import ShardedOCP

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    w = named_workload(args.workload)
    d = synth.draw(w)
    S = ShardedOCP(w, rank=rank, world=world)
    H = S.H
    n, m, nnzj, nnzh = H.n, H.m, H.nnzj, H.nnzh
    sigma = w["sigma"]
    x, y, vn, vm = (torch.from_numpy(d[k]).to(dev) for k in ("x", "y", "vn", "vm"))
    outs = tuple(torch.zeros(k, dtype=torch.float64, device=dev) for k in (1, m, n, nnzj, nnzh, m, n, n))
    flush = L2Flush(dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        S.eval_step(x, y, sigma, vn, vm, outs)

    for _ in range(args.warmup):
        flush()
        step()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(dev.index) if rank == 0 else None
    if sampler:
        sampler.start()
    dist.barrier()
    torch.cuda.synchronize(dev)
    evs = []
    for _ in range(args.steps):
        flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize(dev)
    dist.barrier()
    clocks = sampler.stop() if sampler else None
    tot = torch.tensor([sum(a.elapsed_time(b) for a, b in evs)], dtype=torch.float64, device=dev)
    dist.all_reduce(tot, op=dist.ReduceOp.MAX)
    tot_ms = float(tot.item())
    # end to end: the rank's inputs in (whole arrays: the shard reads its range and a halo) and
    # its owned output slots out, from and to pinned host memory
    hin = [torch.from_numpy(d[k]).pin_memory() for k in ("x", "y", "vn", "vm")]
    din = (x, y, vn, vm)
    slot_of = ("c", "g", "jac", "hess", "c", "g", "g")
    own = [(o, S.owned[sl]) for o, sl in zip(outs[1:], slot_of)]
    hout = [[torch.empty(s1 - s0, dtype=torch.float64).pin_memory() for s0, s1 in sl] for _, sl in own]
    hf = torch.empty(1, dtype=torch.float64).pin_memory()

    def e2e_step():
        for hsrc, dd in zip(hin, din):
            dd.copy_(hsrc, non_blocking=True)
        step()
        for (o, sl), hs in zip(own, hout):
            for (s0, s1), hbuf in zip(sl, hs):
                hbuf.copy_(o[s0:s1], non_blocking=True)
        hf.copy_(outs[0], non_blocking=True)

    e2e_steps = max(3, min(args.steps, 10))
    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize(dev)
    dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2 = torch.tensor([e0.elapsed_time(e1) / e2e_steps], dtype=torch.float64, device=dev)
    dist.all_reduce(e2, op=dist.ReduceOp.MAX)
    nnz = nnzj + nnzh
    res = dict(
        metric=METRIC, value=nnz * args.steps / (tot_ms * 1e-3), unit="nnz/s", n_gpus=world,
        steps=args.steps, warmup=args.warmup, ms_per_step=tot_ms / args.steps, higher_is_better=True,
        scaling="strong", vs_baseline=None, dtype="f64", data="synthetic",
        config=dict(bench_config(args.workload, w, n, m, nnzj, nnzh, world),
                    parallelism="node shards over %d ranks (rank-ordered objective combination)" % world),
        shard=dict(nodes=[S.a, S.b], note="rank 0's node range; each rank runs ocp_eval_step_range on its own"),
        e2e=dict(value=nnz / (float(e2.item()) * 1e-3), unit="nnz/s",
                 h2d_bytes_per_step=sum(8 * t.numel() for t in hin),
                 d2h_bytes_per_step=8 + sum(8 * sum(s1 - s0 for s0, s1 in sl) for _, sl in own),
                 ms=float(e2.item()), note="max over ranks; per rank: whole inputs in, owned slots out"),
        gpu_launches=2 * args.steps, clocks=clocks,
    )
    S.close()
    return res


def run_widened(name, steps, warmup):
    """Fused step, separate calls and J+H alone for one more workload (no e2e, no clocks)."""
    import torch
    from paper_2510_03932_gb300 import ocp

    dev = torch.device("cuda", torch.cuda.current_device())
    w = named_workload(name)
    d = synth.draw(w)
    H = ocp.OCP.from_workload(w)
    x, y, vn, vm = (torch.from_numpy(d[k]).to(dev) for k in ("x", "y", "vn", "vm"))
    sigma = w["sigma"]
    f, c, g, jv, hv, Jv, Jtv, Hv = H.eval_step(x, y, sigma, vn, vm)
    outs = (f, c, g, jv, hv, Jv, Jtv, Hv)
    flush = L2Flush(dev)
    stream = torch.cuda.current_stream(dev)
    calls = {
        "step": lambda: H.eval_step(x, y, sigma, vn, vm, outs),
        "eval_all": lambda: H.eval_all(x, y, sigma, f, c, g, jv, hv, alloc=False),
        "jh": lambda: H.eval_all(x, y, sigma, None, None, None, jv, hv, alloc=False),
        "jprod": lambda: H.jprod(x, vn, Jv),
        "jtprod": lambda: H.jtprod(x, vm, Jtv),
        "hprod": lambda: H.hprod(x, y, sigma, vn, Hv),
    }
    ms = {}
    for nm, fn in calls.items():
        for _ in range(warmup):
            fn()
        evs = []
        for _ in range(steps if nm == "step" else max(3, steps // 4)):
            flush()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize(dev)
        ms[nm] = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    # hot: the same calls without the flush (a problem below the 129 MB L2 then finds part of
    # its inputs and outputs in the cache); labelled, never the reported value.  A short
    # device-side spin before each call (no memory traffic) keeps the GPU busy while the host
    # enqueues the events and the call, as the flush does in the timing above.
    hot = {}
    spin = getattr(torch.cuda, "_sleep", None)   # without it the hot times include launch gaps
    for nm in ("step", "jh"):
        evs = []
        for _ in range(max(3, steps // 4)):
            if spin is not None:
                spin(100000)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            calls[nm]()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize(dev)
        hot[nm + "_ms"] = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    hbm, _ = peaks()
    clk = 2070.0
    fp64_peak = FP64_INST_PER_CLK_PER_SM * NUM_SMS * clk * 1e6 / 1e9
    nnz = H.nnzj + H.nnzh
    out = dict(workload=name, model=w["model"], N=w["N"], n=H.n, m=H.m, nnz_jac=H.nnzj, nnz_hess=H.nnzh,
               step_ms=ms["step"], nnz_per_s=nnz / (ms["step"] * 1e-3),
               separate_calls_ms=ms["eval_all"] + ms["jprod"] + ms["jtprod"] + ms["hprod"],
               jac_hess_only=dict(ms=ms["jh"], nnz_per_s=nnz / (ms["jh"] * 1e-3)), kernels={},
               hot=dict(hot, note="no L2 flush between calls"))
    for nm in ("step", "eval_all", "jh", "jprod", "jtprod", "hprod"):
        ab = algorithmic_bytes(w, nm)
        ops = fp64_ops(ops_model(w), nm)
        out["kernels"][nm] = dict(
            ms=ms[nm], hbm_frac=ab / (ms[nm] * 1e-3) / 1e9 / hbm,
            fp64_frac=(ops * (w["N"] + 1) / (ms[nm] * 1e-3) / 1e9 / fp64_peak) if ops else None)
    out["bound"] = "alu" if (out["kernels"]["step"]["fp64_frac"] or 0) > out["kernels"]["step"]["hbm_frac"] else "hbm"
    out["fp64_peak_basis"] = "2 FP64 inst/clk/SM x 152 SMs x 2070 MHz"
    H.close()
    return out


def run_forms(args, hbm):
    """The batched and differentiation forms, each against the plain evaluator on this GPU."""
    import torch
    from paper_2510_03932_gb300 import autograd as A
    from paper_2510_03932_gb300 import ocp

    out = {}
    # ---- batched: 256 cart-pole instances, N ~ U{500..50000}, one persistent launch in a graph
    ws = synth.batch_workloads()
    probs = [ocp.OCP.from_workload(w) for w in ws]
    B = ocp.OCPBatch(probs)
    draws = [synth.draw(w) for w in ws]
    x = torch.from_numpy(np.concatenate([d["x"] for d in draws])).cuda()
    y = torch.from_numpy(np.concatenate([d["y"] for d in draws])).cuda()
    del draws
    f, c, g, jv, hv = B.outputs()
    best = B.autotune(x, y, 1.0, f, None, g, jv, hv)
    cfg = B.get_config()
    s = torch.cuda.Stream()
    B.graph_capture(x, y, 1.0, f, None, g, jv, hv, stream=s)
    reps = 20
    for _ in range(3):
        B.graph_launch(stream=s)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        B.graph_launch(stream=s)
    e1.record(s)
    s.synchronize()
    t_batch = e0.elapsed_time(e1) / reps
    # the same work as 256 separate plain calls (f, g, J, H per instance)
    xs = [x[B.xoff[i]:B.xoff[i + 1]] for i in range(B.count)]
    ys = [y[B.coff[i]:B.coff[i + 1]] for i in range(B.count)]
    views = [(f[i:i + 1], g[B.xoff[i]:B.xoff[i + 1]], jv[B.joff[i]:B.joff[i + 1]], hv[B.hoff[i]:B.hoff[i + 1]])
             for i in range(B.count)]

    def plain_all():
        for P, xi, yi, (fi, gi, ji, hi) in zip(probs, xs, ys, views):
            P.eval_all(xi, yi, 1.0, fi, None, gi, ji, hi, alloc=False)
    plain_all()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(5):
        plain_all()
    e1.record()
    torch.cuda.synchronize()
    t_plain = e0.elapsed_time(e1) / 5
    nnz = B.nnzj + B.nnzh
    byts = 8 * (B.n + B.m + B.count + B.n + B.nnzj + B.nnzh)
    out["batched"] = dict(workload="256 cart-pole, N~U{500..50000}, seed 1004", total_nodes=int(B.n // 5),
                          nnz=nnz, config=cfg, autotune_best_ms=best, ms=t_batch,
                          nnz_per_s=nnz / (t_batch * 1e-3), GBps=byts / (t_batch * 1e-3) / 1e9,
                          hbm_frac=byts / (t_batch * 1e-3) / 1e9 / hbm,
                          plain_256_calls_ms=t_plain, speedup_vs_plain=t_plain / t_batch,
                          outputs="f, grad, J, H per instance (graph replay of one persistent launch)")
    del B, probs, x, y, f, c, g, jv, hv, xs, ys, views
    torch.cuda.empty_cache()
    # ---- differentiation: c(x; mu) forward + J^T w, (dc/dmu)^T w backward at N = 1e6
    w = synth.workload("vdp_mu_n1e6")
    d = synth.draw(w)
    H = ocp.OCP.from_workload(w)
    xg = torch.from_numpy(d["x"]).cuda().requires_grad_(True)
    mu = torch.tensor([1.0], dtype=torch.float64, device="cuda", requires_grad=True)
    wv = torch.from_numpy(d["vm"]).cuda()

    def ad_step():
        cc = A.constraints(H, xg, mu)
        return torch.autograd.grad(cc, (xg, mu), grad_outputs=wv)

    def plain_step():
        H.eval_cons(xg.detach())
        H.vjp_param(xg.detach(), wv)

    flush = L2Flush("cuda")

    def timed(fn):
        # the same allocator state for every form: collect garbage, then release the caching
        # allocator's free blocks (the preamble torch.cuda.graph runs before a capture).  After a
        # full garbage collection that frees CUDA tensors, this eager step measured 106-127 us
        # instead of 73 us until the cache was emptied; the small problem (N = 2000) and the
        # plain calls showed no such effect.
        gc.collect()
        torch.cuda.empty_cache()
        for _ in range(3):
            fn()
        ts = []
        for _ in range(20):
            flush()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record()
            fn()
            a1.record()
            ts.append((a0, a1))
        torch.cuda.synchronize()
        return float(np.median([a.elapsed_time(b) for a, b in ts]))

    # The eager form and the plain calls first: once torch.cuda.make_graphed_callables has run
    # in a process, PyTorch's eager autograd there is slower (this step: 74 -> 92 us, measured),
    # and a program that trains eagerly builds no graphed callables.
    res = {"autograd": timed(ad_step), "plain": timed(plain_step)}
    # the same autograd step with forward and backward captured in CUDA graphs (the Python
    # and autograd bookkeeping leave the timed path)
    graphed = None
    try:
        gfn = torch.cuda.make_graphed_callables(lambda xx, mm: A.constraints(H, xx, mm), (xg, mu))

        def graphed():
            cc = gfn(xg, mu)
            return torch.autograd.grad(cc, (xg, mu), grad_outputs=wv)
    except Exception as e:  # graph capture unavailable: report the eager form only
        graph_err = "%s: %s" % (type(e).__name__, e)
    # the whole step (forward and backward) captured once in one CUDA graph over the static x,
    # mu and w, as a training loop that replays its step would: no input copy, no Python
    whole = None
    try:
        cs = torch.cuda.Stream()
        cs.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(cs):
            for _ in range(3):
                ad_step()
        torch.cuda.current_stream().wait_stream(cs)
        wg = torch.cuda.CUDAGraph()
        with torch.cuda.graph(wg):
            whole_out = ad_step()   # noqa: F841 (the graph's outputs stay alive with it)
        whole = wg.replay
    except Exception as e:
        whole_err = "%s: %s" % (type(e).__name__, e)
    if graphed:
        res["graphed"] = timed(graphed)
    if whole:
        res["whole_graph"] = timed(whole)
    # the cart-pole's four parameters (m_c, m_p, l, g) as a device tensor: c(x; p) forward and
    # (J^T w, (dc/dp)^T w) backward at N = 1e6, against the same two C-ABI calls made directly
    wc = synth.workload("cartpole_n1e6")
    dc = synth.draw(wc)
    Hc = ocp.OCP.from_workload(wc)
    xc = torch.from_numpy(dc["x"]).cuda().requires_grad_(True)
    pc = torch.tensor(wc["params"], dtype=torch.float64, device="cuda", requires_grad=True)
    wcv = torch.from_numpy(dc["vm"]).cuda()

    def ad_step_p():
        cc = A.constraints(Hc, xc, pc)
        return torch.autograd.grad(cc, (xc, pc), grad_outputs=wcv)

    def plain_step_p():
        Hc.eval_cons_params(xc.detach(), pc.detach())
        Hc.vjp_params(xc.detach(), wcv, pc.detach())

    res_p = {"autograd": timed(ad_step_p), "plain": timed(plain_step_p)}
    out["adjoint_params"] = dict(workload="cartpole_n1e6", step="c(x;p) forward + (J^T w, dc/dp^T w) backward, "
                                 "p = (m_c, m_p, l, g) on the device", autograd_ms=res_p["autograd"],
                                 plain_ms=res_p["plain"], overhead=res_p["autograd"] / res_p["plain"])
    Hc.close()
    del xc, pc, wcv
    out["adjoint"] = dict(workload="vdp_mu_n1e6", step="c(x;mu) forward + (J^T w, dc/dmu^T w) backward",
                          autograd_ms=res["autograd"], plain_ms=res["plain"],
                          overhead=res["autograd"] / res["plain"])
    if "graphed" in res:
        out["adjoint"].update(autograd_graphed_ms=res["graphed"], graphed_overhead=res["graphed"] / res["plain"])
    else:
        out["adjoint"]["graphed_error"] = graph_err
    if "whole_graph" in res:
        out["adjoint"].update(whole_step_graph_ms=res["whole_graph"],
                              whole_step_graph_overhead=res["whole_graph"] / res["plain"],
                              whole_step_graph="forward + backward captured in one CUDA graph over static x, mu, w")
    else:
        out["adjoint"]["whole_step_graph_error"] = whole_err
    return out


def run_profile(args):
    """Few launches of one call, for ncu captures (no timing output of value)."""
    import torch
    from paper_2510_03932_gb300 import ocp

    w = named_workload(args.workload)
    d = synth.draw(w)
    H = ocp.OCP.from_workload(w)
    x, y = torch.from_numpy(d["x"]).cuda(), torch.from_numpy(d["y"]).cuda()
    vn, vm = torch.from_numpy(d["vn"]).cuda(), torch.from_numpy(d["vm"]).cuda()
    f, c, g, jv, hv = H.eval_all(x, y, 1.0)
    Jv, Jtv, Hv = H.jprod(x, vn), H.jtprod(x, vm), H.hprod(x, y, 1.0, vn)
    calls = {
        "eval_all": lambda: H.eval_all(x, y, 1.0, f, c, g, jv, hv, alloc=False),
        "jh": lambda: H.eval_all(x, y, 1.0, None, None, None, jv, hv, alloc=False),
        "jprod": lambda: H.jprod(x, vn, Jv),
        "jtprod": lambda: H.jtprod(x, vm, Jtv),
        "hprod": lambda: H.hprod(x, y, 1.0, vn, Hv),
        "step": lambda: H.eval_step(x, y, 1.0, vn, vm, (f, c, g, jv, hv, Jv, Jtv, Hv)),
    }
    if args.profile_kernel == "kkt":  # KKT assembly from this H and J (sigma_x = 1)
        sx = torch.ones(H.n, dtype=torch.float64, device="cuda")
        kv = H.kkt_values(hv, jv, sx, 1e-8, 1e-8)
        calls = {"kkt": lambda: H.kkt_values(hv, jv, sx, 1e-8, 1e-8, out=kv)}
    fns = list(calls.values()) if args.profile_kernel == "all" else [calls[args.profile_kernel]]
    for _ in range(args.warmup + args.steps):
        for fn in fns:
            fn()
    torch.cuda.synchronize()
    print(json.dumps(dict(profile_kernel=args.profile_kernel, workload=args.workload, launches=args.warmup + args.steps)))


def oracle_step_time(w, budget_s):
    """Time the oracle on a bounded sample of the workload: the same problem at a shorter
    horizon, evaluated in full (values, products) as many times as fit in budget_s."""
    from oracle import oracle as O
    Ns = min(w["N"], 100000)
    ws = synth.with_horizon(w, Ns)
    d = synth.draw(ws)
    P = O.Problem(ws)
    reps, t0 = 0, time.perf_counter()
    while True:
        O.evaluate(P, d["x"], d["y"], ws["sigma"])
        O.jprod(P, d["x"], d["vn"])
        O.jtprod(P, d["x"], d["vm"])
        O.hprod(P, d["x"], d["y"], ws["sigma"], d["vn"])
        reps += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = (time.perf_counter() - t0) / reps
    return (P.nnzj + P.nnzh) / dt, dict(value=(P.nnzj + P.nnzh) / dt, unit="nnz/s", cores=1, kind="oracle",
                                        sample="%s at N=%d (full step: eval + 3 products), %d reps, %.1f s"
                                               % (w["name"], Ns, reps, reps * dt))


def _oracle_worker(args):
    """One host core: the oracle step on its own node shard (a problem of Ns nodes)."""
    w, Ns, budget_s = args
    sys.path.insert(0, ROOT)
    _, info = oracle_step_time(synth.with_horizon(w, Ns), budget_s)
    return info["value"]


def oracle_parallel(w, budget_s, cores=None, pool=None, rounds=1):
    """The oracle on every host core at once: each process evaluates its own shard of Ns nodes
    (the node loops split across cores, as the loops of a node-parallel CPU code would be);
    throughput = sum over the processes, one value per round.  Spawned processes (no fork
    after CUDA use)."""
    import multiprocessing as mp
    cores = cores or len(os.sched_getaffinity(0))
    Ns = min(w["N"], 100000)
    own = pool is None
    if own:
        pool = mp.get_context("spawn").Pool(cores)
    try:
        vals = [float(sum(pool.map(_oracle_worker, [(w, Ns, budget_s)] * cores))) for _ in range(rounds)]
    finally:
        if own:
            pool.close()
            pool.join()
    return (vals[0] if rounds == 1 else vals), cores, Ns


def _free_port():
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--no-forms", action="store_true", help="skip the batched and differentiation forms")
    ap.add_argument("--shard", action="store_true",
                    help="split ONE problem over the ranks (node shards, strong scaling) instead of replicas")
    ap.add_argument("--no-widened", action="store_true", help="skip the further workloads (quadrotor, Goddard)")
    ap.add_argument("--profile-kernel", default=None,
                    choices=["eval_all", "jh", "jprod", "jtprod", "hprod", "step", "kkt", "all"],
                    help="only launch this call warmup+steps times (for ncu captures)")
    args = ap.parse_args()
    if args.profile_kernel:
        run_profile(args)
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        if rank != 0:
            return
        w = named_workload(args.workload)
        # the oracle on every host core: one process per core, each on its own node shard;
        # one warm-up round, then one bounded round per step
        budget = max(1.0, args.cpu_budget / max(1, args.steps))
        vals, cores, Ns = oracle_parallel(w, budget, rounds=args.steps + (1 if args.warmup > 0 else 0))
        vals = vals if isinstance(vals, list) else [vals]
        if args.warmup > 0 and len(vals) > 1:
            vals = vals[1:]
        v = float(np.mean(vals))
        cb = dict(value=v, unit="nnz/s", cores=cores, kind="oracle",
                  sample="%s: %d processes, each the full step (eval + 3 products) on its own %d-node shard, "
                         "%.1f s per step" % (w["name"], cores, Ns, budget))
        from oracle import oracle as O
        P = O.Problem(w)
        nnz = P.nnzj + P.nnzh
        print(json.dumps(dict(metric=METRIC, value=v, unit="nnz/s", n_gpus=1, steps=args.steps, warmup=args.warmup,
                              # the time one step of the whole workload takes at the sampled rate
                              ms_per_step=nnz / v * 1e3, higher_is_better=True, scaling="weak", vs_baseline=None,
                              impl="reference", dtype="f64", data="synthetic",
                              config=bench_config(args.workload, w, P.n, P.m, P.nnzj, P.nnzh, 1),
                              cpu_baseline=cb, e2e=dict(value=v, unit="nnz/s", h2d_bytes_per_step=0,
                                                        d2h_bytes_per_step=0))))
        return
    if args.shard:
        import torch
        if world == 1 and "MASTER_ADDR" not in os.environ:
            os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()), RANK="0", WORLD_SIZE="1")
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0))))
        res = run_sharded(args, rank, world)
        if rank == 0:
            print(json.dumps(res))
        torch.distributed.destroy_process_group()
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    res = run_ours(args, rank, world)
    if rank == 0 and not args.no_forms:
        res["forms"] = run_forms(args, res["roofline_hbm"]["peak"])
    if rank == 0 and not args.no_widened:
        res["configs"] = {nm: run_widened(nm, min(args.steps, 200), max(args.warmup, 3)) for nm in CONFIGS}
        res["widened"] = {nm: run_widened(nm, min(args.steps, 200), max(args.warmup, 3)) for nm in WIDENED
                          if nm != args.workload}
    if rank == 0:
        wl = named_workload(args.workload)
        _, single = oracle_step_time(wl, args.cpu_budget / 2)
        par, cores, Ns = oracle_parallel(wl, args.cpu_budget / 2)
        res["cpu_baseline"] = dict(value=par, unit="nnz/s", cores=cores, kind="oracle",
                                   sample="%s: %d processes, each the full step (eval + 3 products) on its own "
                                          "%d-node shard for %.1f s" % (wl["name"], cores, Ns, args.cpu_budget / 2),
                                   single_core=single)
        print(json.dumps(res))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
