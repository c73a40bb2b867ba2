"""The Goddard kernels' table-driven exponential (x = (32 m + j) ln 2/32 + r, 2^(j/32) from a
table, a degree-6 polynomial in r, 2^m on the exponent bits; the library routine for warps
holding an argument beyond 700 in magnitude or not finite) against numpy and CUDA's exp within
two ulps, on uniform, wide and table-edge samples; exp(0) = 1 exactly; the library's own values
on the fallback path."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def probe():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2510_03932_gb300 import ocp
    return ocp.probe_exp


def ulps(got, ref):
    return np.abs(got - ref) / np.spacing(np.maximum(np.abs(ref), 2.0 ** -1022))


def run(probe, x):
    outs = probe(torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda())
    return [o.cpu().numpy() for o in outs]


def test_within_two_ulps(probe):
    rng = np.random.default_rng(17)
    x = np.concatenate([rng.uniform(-1.0, 1.0, 200000), rng.uniform(-20.0, 0.0, 200000),   # the drag term's range
                        rng.uniform(-700.0, 700.0, 100000), 10.0 ** rng.uniform(-300.0, 2.0, 50000),
                        (np.arange(-20000, 20000) + 0.5) * (np.log(2) / 32),                  # table edges
                        np.arange(-20000, 20000) * (np.log(2) / 32)])
    e, el = run(probe, x)
    for ref in (np.exp(x), el):
        err = ulps(e, ref)
        assert err.max() <= 2.0, (err.max(), x[np.argmax(err)])


def test_exact_cases(probe):
    e, _ = run(probe, np.array([0.0, -0.0, 5e-324, -5e-324, 1e-300, -1e-300]))
    assert np.all(e == 1.0)


def test_fallback_warps_take_the_library_values(probe):
    rng = np.random.default_rng(23)
    x = rng.uniform(-5.0, 5.0, 32 * 16)
    x[::64] = 705.0          # one lane in every other warp (still finite: exp(705) < DBL_MAX)
    x[32 * 5 + 3] = -800.0   # underflows to a subnormal in the library routine
    x[32 * 7 + 1] = np.nan
    e, el = run(probe, x)
    for w in range(16):
        sel = slice(32 * w, 32 * w + 32)
        if w % 2 == 0 or w in (5, 7):
            assert np.array_equal(e[sel], el[sel], equal_nan=True)
        else:
            assert ulps(e[sel], el[sel]).max() <= 2.0
