"""The tables of the kernels' table-driven sine and cosine (csrc/sincos_table_data.h) and
exponential (csrc/exp_table_data.h) and the constants of their argument reductions
(csrc/sincos_table.cuh, csrc/exp_table.cuh), pinned to the mathematics: every entry is the
double nearest sin(i pi/512), cos(i pi/512) or 2^(j/32) (mpmath at 60 digits), the quadrant
symmetry sin(i pi/512) = cos((256 - i) pi/512) holds entry for entry, 2^(16/32) is the nearest
double to sqrt(2), and the splits of pi/512 and ln 2/32 and the constants 512/pi and 32/ln 2
are the doubles nearest the exact values."""
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


def exp_table():
    src = open(os.path.join(CSRC, "exp_table_data.h")).read()
    rows = [float.fromhex(a) for a in re.findall(r"^\s+(\S+),  //", src, re.M)]
    assert len(rows) == 32
    return np.array(rows)


def test_exp_table_shape():
    t = exp_table()
    assert t[0] == 1.0 and t[16] == float(np.sqrt(2.0))       # 2^0 and 2^(1/2), both the nearest doubles
    assert np.all(np.diff(t) > 0) and t[-1] < 2.0
    # 2^(j/32) 2^((32-j)/32) = 2 to within the two roundings
    assert np.max(np.abs(t[1:] * t[:0:-1] - 2.0)) <= 4 * np.finfo(float).eps


def test_exp_entries_are_the_nearest_doubles():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    for j, v in enumerate(exp_table()):
        exact = mpmath.power(2, mpmath.mpf(j) / 32)
        assert abs(mpmath.mpf(v) - exact) <= mpmath.mpf(np.spacing(v)) / 2, j


def test_exp_reduction_constants():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    src = open(os.path.join(CSRC, "exp_table.cuh")).read()
    inv = float.fromhex(re.search(r"fma\(x, (\S+), 0x1\.8p52\);\s+// 32 / ln 2", src).group(1))
    parts = [float.fromhex(m) for m in re.findall(r"r = fma\(-k, (\S+), (?:x|r)\);\s+// L\d", src)]
    assert len(parts) == 2
    assert inv == float(32 / mpmath.log(2))
    exact = mpmath.log(2) / 32
    assert parts[0] == float(exact) and parts[1] == float(exact - parts[0])
    # the series coefficients 1/n! for n = 2..6 are the doubles nearest 1/n!
    for n, pat in ((6, r"fma\(r, (\S+), \S+\);\s+// 1/6!"), (5, r"fma\(r, \S+, (\S+)\);\s+// 1/6!, 1/5!"),
                   (4, r"fma\(r, q, (\S+)\);\s+// 1/4!"), (3, r"fma\(r, q, (\S+)\);\s+// 1/3!")):
        c = float.fromhex(re.search(pat, src).group(1))
        assert c == float(1 / mpmath.factorial(n)), n
