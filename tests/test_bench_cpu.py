"""The benchmark's measurement arithmetic and its reference arm, on the CPU: the algorithmic
bytes behind the HBM roofline, the FP64 peak, the FP64 instruction table's coverage of every
reported workload, and the JSON line of `bench.py --impl reference` (the oracle on host cores)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2510_03932_gb300 import synth  # noqa: E402


def test_algorithmic_bytes_of_the_headline_workload(monkeypatch):
    """Van der Pol (mu), N = 1e6: n = 3N+3, m = 2N+2, nnz_J = 10N+2, nnz_H = 4(N+1); J + H moves
    each input and output once (152 MB), the fused step its twelve arrays (296 MB)."""
    w = bench.named_workload("vdp_mu_n1e6")
    N = w["N"]
    P = O.Problem(w)
    assert (P.n, P.m, P.nnzj, P.nnzh) == (3 * N + 3, 2 * N + 2, 10 * N + 2, 4 * (N + 1))
    monkeypatch.setattr(bench, "_counts", lambda ww: (P.nnzj, P.nnzh))
    n, m = P.n, P.m
    assert bench.algorithmic_bytes(w, "jh") == 8 * (n + m + P.nnzj + P.nnzh) == 152_000_088
    # reads x, y, vn, vm (2n + 2m); writes f, c, g, J, H, Jv, J^T w, Hv (1 + 2m + 3n + nnz)
    assert bench.algorithmic_bytes(w, "step") == 8 * (5 * n + 4 * m + 1 + P.nnzj + P.nnzh)
    assert bench.algorithmic_bytes(w, "step") == 296_000_240
    assert bench.algorithmic_bytes(w, "jprod") == 8 * (2 * n + m)
    with pytest.raises(KeyError):
        bench.algorithmic_bytes(w, "nothing")


def test_fp64_peak_from_unit_counts():
    """2 FP64 instructions per clock per SM x 152 SMs x 2070 MHz = 629.28 G instructions/s."""
    assert bench.FP64_INST_PER_CLK_PER_SM * bench.NUM_SMS * 2070e6 / 1e9 == pytest.approx(629.28)


def test_fp64_counts_are_tagged_with_the_kernel_sources_they_were_measured_on():
    """Every measured FP64-instruction count and DRAM-traffic figure carries the tag of the
    kernel sources it was measured on; a change to those sources without a new measurement
    (and a new tag) fails here, so the bench can never divide by a stale count silently."""
    for key, tag in bench.FP64_OPS_SRC.items():
        assert bench.kernel_source_tag(key) == tag, (
            "kernel sources of %r changed since its FP64 counts were measured: re-measure them "
            "(profiles/fp64_ops_per_node.md) and update FP64_OPS_SRC" % key)
    for (name, kern), (_, tag) in bench.TRAFFIC.items():
        key = bench.ops_model(bench.named_workload(name))
        assert bench.kernel_source_tag(key) == tag, (name, kern)


def test_stale_counts_are_not_used(monkeypatch):
    monkeypatch.setitem(bench.FP64_OPS_SRC, "vdp", "000000000000")
    assert bench.fp64_ops("vdp", "step") is None
    monkeypatch.setitem(bench.TRAFFIC, ("vdp_mu_n1e6", "step"), (1.0, "000000000000"))
    assert bench.traffic("vdp_mu_n1e6", "step", "vdp") is None


def test_fp64_table_covers_every_reported_workload():
    names = ["vdp_mu_n1e6"] + bench.WIDENED + bench.CONFIGS
    for name in names:
        key = bench.ops_model(bench.named_workload(name))
        for kern in ("step", "eval_all", "jh", "jprod", "jtprod", "hprod"):
            assert (key, kern) in bench.FP64_OPS_PER_NODE, (name, kern)
    # the fused step never costs more than its four separate calls
    for (model, kern), ops in bench.FP64_OPS_PER_NODE.items():
        if kern == "step":
            parts = sum(bench.FP64_OPS_PER_NODE[(model, k)] for k in ("eval_all", "jprod", "jtprod", "hprod"))
            assert ops <= parts + 1e-9, model


def _run(args, env=None, timeout=300):
    e = dict(os.environ, **(env or {}))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, capture_output=True, text=True,
                       timeout=timeout, cwd=ROOT, env=e)
    return r


def test_reference_arm_prints_the_contract_line():
    r = _run(["--impl", "reference", "--workload", "vdp_n1e3", "--steps", "1", "--warmup", "0", "--cpu-budget", "1"])
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "nnz/s" and d["value"] > 0 and d["dtype"] == "f64"
    assert d["config"]["workload"] == "vdp_n1e3" and d["config"]["nnz_jac"] == 10 * 1000 + 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == dict(value=d["value"], unit="nnz/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0)
    # the same config object as the GPU arm's line
    w = bench.named_workload("vdp_n1e3")
    P = O.Problem(w)
    assert d["config"] == bench.bench_config("vdp_n1e3", w, P.n, P.m, P.nnzj, P.nnzh, 1)


def test_reference_arm_other_ranks_exit_quietly():
    r = _run(["--impl", "reference", "--workload", "vdp_n1e3", "--steps", "1", "--warmup", "0", "--cpu-budget", "1"],
             env={"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0 and r.stdout.strip() == ""
