"""The table of the kernels' table-driven sine and cosine (csrc/sincos_table_data.h) and the
constants of its argument reduction (csrc/sincos_table.cuh), pinned to the mathematics:
every entry is the double nearest sin(i pi/512) or cos(i pi/512) (mpmath at 60 digits), the
quadrant symmetry sin(i pi/512) = cos((256 - i) pi/512) holds entry for entry, and the
three-part split of pi/512 and the constant 512/pi are the doubles nearest the exact values."""
import os
import re

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2510_03932_gb300", "csrc")


def table():
    src = open(os.path.join(CSRC, "sincos_table_data.h")).read()
    rows = [(float.fromhex(a), float.fromhex(b)) for a, b in re.findall(r"\{(\S+), (\S+)\},", src)]
    assert len(rows) == 256
    return np.array(rows)


def test_symmetry_and_unit_circle():
    t = table()
    assert t[0, 0] == 0.0 and t[0, 1] == 1.0
    for i in range(1, 256):
        assert t[i, 0] == t[256 - i, 1]   # sin(i pi/512) = cos((256-i) pi/512): the same nearest double
    r = t[:, 0] ** 2 + t[:, 1] ** 2
    assert np.max(np.abs(r - 1.0)) <= 4 * np.finfo(float).eps
    # increasing sine, decreasing cosine on [0, pi/2)
    assert np.all(np.diff(t[:, 0]) > 0) and np.all(np.diff(t[:, 1]) < 0)


def test_entries_are_the_nearest_doubles():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    t = table()
    for i in range(256):
        a = mpmath.mpf(i) * mpmath.pi / 512
        for v, exact in ((t[i, 0], mpmath.sin(a)), (t[i, 1], mpmath.cos(a))):
            err = abs(mpmath.mpf(v) - exact)
            half_ulp = mpmath.mpf(np.spacing(abs(v)) if v != 0 else 0) / 2
            assert err <= half_ulp, (i, v)


def test_reduction_constants():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    src = open(os.path.join(CSRC, "sincos_table.cuh")).read()
    inv = float.fromhex(re.search(r"fma\(ax, (\S+), 0x1\.8p52\);\s+// 512/pi", src).group(1))
    p = [float.fromhex(m) for m in re.findall(r"r = fma\(-k, (\S+), (?:ax|r)\);\s+// P\d", src)]
    assert len(p) == 3
    assert inv == float(512 / mpmath.pi)
    exact = mpmath.pi / 512
    # each part is the double nearest what the previous parts leave of pi/512
    assert p[0] == float(exact)
    assert p[1] == float(exact - p[0])
    assert p[2] == float(exact - p[0] - p[1])
    assert abs(exact - (mpmath.mpf(p[0]) + p[1] + p[2])) < mpmath.mpf(2) ** -170
