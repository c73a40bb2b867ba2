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


def _fma(a, b, c):
    """a * b + c with one rounding (exact rational arithmetic, then the nearest double)."""
    from fractions import Fraction
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _hexes(pattern, src, count):
    found = [float.fromhex(m) for m in re.findall(pattern, src)]
    assert len(found) == count, (pattern, found)
    return found


def test_sincos_method_within_two_ulps_on_the_cpu():
    """The table-driven sin and cos, replayed step by step on the CPU with the constants and table
    of the committed sources (each FMA rounded once), stay within two ulps of the exact values
    (mpmath) on a sample that covers small, large, near-multiple-of-pi/2 and table-edge arguments."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    src = open(os.path.join(CSRC, "sincos_table.cuh")).read()
    inv = _hexes(r"fma\(ax, (\S+), 0x1\.8p52\);\s+// 512/pi", src, 1)[0]
    p1, p2, p3 = _hexes(r"r = fma\(-k, (\S+), (?:ax|r)\);\s+// P\d", src, 3)
    HEX = r"(-?0x[0-9a-f.]+p[-+]\d+)"
    m = re.search(r"fma\(z, " + HEX + ", " + HEX + r"\), r\);\s+// 1/5!, -1/3!", src)
    c5, c3 = float.fromhex(m.group(1)), float.fromhex(m.group(2))
    c4 = float.fromhex(re.search(r"fma\(z, " + HEX + r", -0\.5\)\);\s+// 1/4!, -1/2!", src).group(1))
    assert (c5, c3, c4) == (1 / 120, -1 / 6, 1 / 24)
    tab = table()
    C52 = 1.5 * 2.0 ** 52

    def sincos(x):
        ax = abs(x)
        t = _fma(ax, inv, C52)
        k = _fma(-C52, 1.0, t)
        r = _fma(-k, p1, ax); r = _fma(-k, p2, r); r = _fma(-k, p3, r)
        ki = int(k)
        sa, ca = tab[ki & 255]
        z = _fma(r, r, -0.0)
        sr = _fma(_fma(r, z, -0.0), _fma(z, c5, c3), r)
        cm1 = _fma(z, _fma(z, c4, -0.5), -0.0)
        sy = _fma(ca, sr, _fma(sa, cm1, sa))
        cy = _fma(-sa, sr, _fma(ca, cm1, ca))
        q = (ki >> 8) & 3
        s, c = [(sy, cy), (cy, -sy), (-sy, -cy), (-cy, sy)][q]
        return (s if x >= 0 else -s), c

    rng = np.random.default_rng(29)
    k = rng.integers(-60000, 60000, 300)
    xs = np.concatenate([rng.uniform(-1, 1, 400), rng.uniform(-1e5, 1e5, 300), 10.0 ** rng.uniform(-300, 5, 200),
                         k * (np.pi / 2) + rng.uniform(-1e-6, 1e-6, k.size),
                         (rng.integers(-4000, 4000, 400) + 0.5) * (np.pi / 512)])
    xs = xs[np.abs(xs) <= 1e5]
    for x in xs:
        s, c = sincos(float(x))
        es, ec = mpmath.sin(float(x)), mpmath.cos(float(x))
        for got, exact in ((s, es), (c, ec)):
            ref = float(exact)
            assert abs(mpmath.mpf(got) - exact) <= 2 * np.spacing(max(abs(ref), 2.0 ** -1022)), (x, got, ref)


def test_exp_method_within_one_ulp_on_the_cpu():
    """The table-driven exponential, replayed step by step on the CPU with the constants and table
    of the committed sources, stays within one ulp of the exact value (mpmath)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    src = open(os.path.join(CSRC, "exp_table.cuh")).read()
    inv = float.fromhex(re.search(r"fma\(x, (\S+), 0x1\.8p52\);\s+// 32 / ln 2", src).group(1))
    l1, l2 = _hexes(r"r = fma\(-k, (\S+), (?:x|r)\);\s+// L\d", src, 2)
    c6 = float.fromhex(re.search(r"fma\(r, (\S+), \S+\);\s+// 1/6!", src).group(1))
    c5 = float.fromhex(re.search(r"fma\(r, \S+, (\S+)\);\s+// 1/6!, 1/5!", src).group(1))
    c4 = float.fromhex(re.search(r"fma\(r, q, (\S+)\);\s+// 1/4!", src).group(1))
    c3 = float.fromhex(re.search(r"fma\(r, q, (\S+)\);\s+// 1/3!", src).group(1))
    tab = exp_table()
    C52 = 1.5 * 2.0 ** 52

    def ex(x):
        t = _fma(x, inv, C52)
        k = _fma(-C52, 1.0, t)
        r = _fma(-k, l1, x); r = _fma(-k, l2, r)
        ki = int(k)
        q = _fma(r, c6, c5); q = _fma(r, q, c4); q = _fma(r, q, c3); q = _fma(r, q, 0.5)
        p = _fma(_fma(r, r, -0.0), q, r)
        tj = tab[ki & 31]
        return _fma(tj, p, tj) * 2.0 ** (ki >> 5)

    rng = np.random.default_rng(31)
    xs = np.concatenate([rng.uniform(-1, 1, 400), rng.uniform(-20, 0, 400), rng.uniform(-700, 700, 300),
                         (rng.integers(-20000, 20000, 300) + 0.5) * (np.log(2) / 32)])
    for x in xs:
        got, exact = ex(float(x)), mpmath.exp(float(x))
        assert abs(mpmath.mpf(got) - exact) <= np.spacing(float(exact)), (x, got)
