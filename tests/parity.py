"""Shared helpers of the parity tests: the tolerance gate and oracle/GPU plumbing.

Gate (per entry): |gpu - oracle| <= 1e-12 |oracle| + 1e-14, or, for entries whose value
suffers cancellation, |gpu - oracle| <= 1e-12 * shadow, where shadow is the oracle's
running-error magnitude of the same expression (the sum of the magnitudes of the terms).
Entries passing only through the second clause are counted and reported.
"""
import numpy as np

RTOL = 1e-12
ATOL = 1e-14


def gate(name, gpu, ref, shadow=None, report=None):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert gpu.shape == ref.shape, (name, gpu.shape, ref.shape)
    err = np.abs(gpu - ref)
    ok1 = err <= RTOL * np.abs(ref) + ATOL
    ok = ok1.copy()
    if shadow is not None:
        ok |= err <= RTOL * np.asarray(shadow)
    bad = np.where(~ok)[0]
    if report is not None:
        report[name] = dict(n=int(ref.size), cancellation=int(np.sum(ok & ~ok1)), fail=int(bad.size),
                            max_rel=float(np.max(err / np.maximum(np.abs(ref), 1e-300))) if ref.size else 0.0)
    if bad.size:
        i = bad[0]
        raise AssertionError("%s: %d of %d entries outside the gate; first at %d: gpu=%r oracle=%r shadow=%r"
                             % (name, bad.size, ref.size, i, gpu[i], ref[i],
                                None if shadow is None else np.asarray(shadow)[i]))
