"""The evaluation kernels' two sin and cos routines against numpy within two ulps and CUDA's
sincos within three, on uniform, log-uniform, near-multiple-of-pi/2 and table-edge samples;
exact zeros and signs where the result is exact; the library's own values on the fallback
path.  The routines: a three-constant Cody-Waite reduction to |r| <= pi/4 with Taylor
polynomials of sin r through r^17 and cos r through r^16 (ocp_probe_sincos), and the
table-driven one of the cart-pole and quadrotor models, |x| = k pi/512 + r with sin, cos of
k pi/512 from a table and short polynomials in r (ocp_probe_sincos_table); both take the
library routine for warps holding an argument beyond 1e5 or not finite."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=[False, True], ids=["reduced", "table"])
def probe(request):
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2510_03932_gb300 import ocp
    return lambda x: ocp.probe_sincos(x, table=request.param)


def ulps(got, ref):
    """|got - ref| in units of the last place of ref (at least that of 2^-1022)."""
    return np.abs(got - ref) / np.spacing(np.maximum(np.abs(ref), 2.0 ** -1022))


def run(probe, x):
    outs = probe(torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda())
    return [o.cpu().numpy() for o in outs]


def test_within_two_ulps(probe):
    rng = np.random.default_rng(11)
    k = rng.integers(-60000, 60000, 100000)
    x = np.concatenate([rng.uniform(-1.0, 1.0, 200000), rng.uniform(-7.0, 7.0, 200000),
                        rng.uniform(-1e5, 1e5, 100000), 10.0 ** rng.uniform(-300.0, 5.0, 100000),
                        k * (np.pi / 2) + rng.uniform(-1e-6, 1e-6, k.size),   # near multiples of pi/2
                        np.arange(-64, 65) * (np.pi / 4),
                        (np.arange(-4096, 4096) + 0.5) * (np.pi / 512),          # table edges
                        (np.arange(-4096, 4096) + rng.uniform(-0.5, 0.5, 8192)) * (np.pi / 512)])
    x = x[np.abs(x) <= 1e5]
    s, c, sl, cl = run(probe, x)
    # against numpy (glibc: correctly rounded or within an ulp) and against CUDA's sincos
    for got, ref, bound in ((s, np.sin(x), 2.0), (c, np.cos(x), 2.0), (s, sl, 3.0), (c, cl, 3.0)):
        e = ulps(got, ref)
        assert e.max() <= bound, (e.max(), x[np.argmax(e)])


def test_exact_cases_and_signs(probe):
    tiny = np.array([0.0, -0.0, 5e-324, -5e-324, 1e-300, -1e-300, 1e-17, -1e-17])
    s, c, sl, cl = run(probe, tiny)
    assert np.array_equal(s, tiny) and np.array_equal(np.signbit(s), np.signbit(tiny))
    assert np.all(c == 1.0)


def test_fallback_warps_take_the_library_values(probe):
    """A warp with one argument beyond 1e5 (or not finite) computes every lane with CUDA's
    sincos; a warp of small arguments does not need to."""
    rng = np.random.default_rng(5)
    x = rng.uniform(-3.0, 3.0, 32 * 64)
    x[::64] = 1e7          # one lane in every other warp
    x[32 * 5 + 3] = np.nan
    x[32 * 9 + 7] = np.inf
    s, c, sl, cl = run(probe, x)
    for w in range(64):
        sel = slice(32 * w, 32 * w + 32)
        if w % 2 == 0 or w in (5, 9):
            assert np.array_equal(s[sel], sl[sel], equal_nan=True) and np.array_equal(c[sel], cl[sel], equal_nan=True)
        else:
            assert ulps(s[sel], sl[sel]).max() <= 2.0 and ulps(c[sel], cl[sel]).max() <= 2.0
    assert np.isnan(s[32 * 5 + 3]) and np.isnan(c[32 * 9 + 7])
