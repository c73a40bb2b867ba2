"""The evaluation kernels' reciprocal (Newton-Raphson steps from the hardware's approximate
reciprocal, used for the cart-pole's 1/D, the quadrotor's 1/cos x8 and the Goddard rocket's
1/m and 1/r) against the IEEE division: within one ulp of the correctly rounded 1/d over a
log-uniform sample of normal doubles of both signs, and exact on powers of two."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_recip_within_one_ulp_of_ieee_division():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2510_03932_gb300 import ocp
    rng = np.random.default_rng(7)
    e = rng.uniform(-300.0, 300.0, 400000)
    d = np.concatenate([10.0 ** e * rng.choice([-1.0, 1.0], e.size), rng.uniform(0.5, 2.0, 200000),
                        rng.uniform(1.0, 1.02, 50000), np.cos(rng.uniform(-1.0, 1.0, 50000)),
                        2.0 ** np.arange(-1000, 1001, dtype=np.float64)])
    got = ocp.probe_recip(torch.from_numpy(d).cuda()).cpu().numpy()
    ref = 1.0 / d
    ulp = np.spacing(np.abs(ref))
    err = np.abs(got - ref) / ulp
    assert np.all(np.isfinite(got))
    assert err.max() <= 1.0, (err.max(), d[np.argmax(err)])
    pow2 = d[-2001:]
    assert np.array_equal(got[-2001:], 1.0 / pow2)
