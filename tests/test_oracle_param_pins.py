"""Pins of the oracle's parameter derivatives (dc/dp)^T w for every dynamics parameter (no GPU).

Each model's df/dp is written out by hand in the oracle; here it is checked against
  - the complex-step derivative of the constraint residual in each parameter (a derivative of
    the right-hand side the oracle evaluates, not of the hand-written df/dp);
  - scaling laws of the equations of motion, which tie the parameter derivatives to the
    Jacobian's control column and to the constraint values:
      cart-pole: f is unchanged when (mc, mp, F) scale together, and the cart's acceleration
      scales with (l, g, F) while the pole's angular acceleration does not;
      Goddard:   thrust enters as u Tmax, and m' is linear in b;
      quadrotor: g enters x6' alone, with coefficient -1 (a closed form for (dc/dg)^T w).
A dropped term, a wrong sign or a swapped parameter in any df/dp fails one of these.
"""
import numpy as np
import pytest

from oracle import oracle as O
from test_oracle_pins import rand_point, small

WITH_PARAMS = ["vdp_n1e3", "cartpole_n1e5", "goddard_n1e3", "quadrotor_n1e3", "vdp_n1e3:euler",
               "cartpole_n1e5:euler", "quadrotor_n1e3:euler", "cartpole_n1e5+path", "goddard_n1e3+path"]
NPAR = {"vdp": 1, "cartpole": 4, "goddard": 4, "quadrotor": 1, "dint": 0, "heat": 0}


def point(name, N, seed):
    w = small(name, N)
    P = O.Problem(w)
    rng = np.random.default_rng(seed)
    x, _ = rand_point(w, rng)
    return w, P, x, rng.standard_normal(P.m)


def defect_row(P, w, k, j):
    """Row of defect (k, j): the boundary rows come first, then N defects per component."""
    nb = P.m - w["nx"] * w["N"] - (len(w["path"]["r"]) * (w["N"] + 1) if w.get("path") else 0)
    return nb + k * w["N"] + j


@pytest.mark.parametrize("name", WITH_PARAMS)
def test_dpar_all_vs_complex_step(name):
    w, P, x, wv = point(name, 23, 5)
    assert O.npar(P) == NPAR[w["model"]]
    got, mag = O.dpar_vjp_all(P, x, wv, shadow=True)
    for i in range(O.npar(P)):
        ref = wv @ O.cs_cons_p(P, x, np.zeros(P.n), np.eye(O.npar(P))[i])
        assert abs(got[i] - ref) <= 1e-13 * mag[i] + 1e-300, (name, i, got[i], ref)
        assert mag[i] >= abs(got[i])


def test_dpar_all_agrees_with_the_mu_derivative():
    w, P, x, wv = point("vdp_n1e3", 40, 9)
    assert O.dpar_vjp_all(P, x, wv)[0] == O.dpar_vjp(P, x, wv)


@pytest.mark.parametrize("name", ["dint", "heat_n2e4"])
def test_models_without_parameter_derivatives(name):
    w, P, x, wv = point(name, 7, 1)
    assert O.npar(P) == 0
    with pytest.raises(RuntimeError):
        O.dpar_vjp_all(P, x, wv)


@pytest.mark.parametrize("scheme", ["", ":euler"])
def test_quadrotor_gravity_closed_form(scheme):
    """x6' = u1 R - g: dc_{5,j}/dg = h (trapezoid: h (1 + 1) / 2; Euler: h) on the x6 defects."""
    name = "quadrotor_n1e3" + scheme
    w, P, x, wv = point(name, 31, 3)
    h = w["T"] / w["N"]
    expect = h * sum(wv[defect_row(P, w, 5, j)] for j in range(w["N"]))
    got = O.dpar_vjp_all(P, x, wv)[0]
    assert abs(got - expect) <= 1e-13 * h * np.abs(wv).sum()


def test_cartpole_scaling_laws():
    """With F the control column and c1 the cart-acceleration defects:
      mc dc/dmc + mp dc/dmp + sum_j F_j dc/dF_j = 0                     (f is degree 0 in (mc, mp, F))
      l dc/dl + g dc/dg + sum_j F_j dc/dF_j = (defect part of c_1)       (pdd degree 1, thdd degree 0
                                                                          in (l, g, F))
    contracted with w; the Jacobian's F column comes from the oracle's J^T w."""
    w, P, x, wv = point("cartpole_n1e5", 29, 11)
    mc, mp, l, g = w["params"]
    N, nx = w["N"], w["nx"]
    d = O.dpar_vjp_all(P, x, wv)
    Jtw = O.jtprod(P, x, wv)
    F = x[nx * (N + 1):nx * (N + 1) + N + 1]
    fterm = F @ Jtw[nx * (N + 1):nx * (N + 1) + N + 1]
    scale = abs(mc * d[0]) + abs(mp * d[1]) + abs(fterm) + abs(l * d[2]) + abs(g * d[3])
    assert abs(mc * d[0] + mp * d[1] + fterm) <= 1e-12 * scale
    c = O.evaluate(P, x, np.zeros(P.m), 1.0)["c"]
    X = x[:nx * (N + 1)].reshape(N + 1, nx)
    rows = [defect_row(P, w, 1, j) for j in range(N)]
    rhs = sum(wv[r] * (c[r] - (X[j + 1, 1] - X[j, 1])) for j, r in enumerate(rows))
    assert abs(l * d[2] + g * d[3] + fterm - rhs) <= 1e-12 * (scale + abs(rhs))


def test_goddard_thrust_and_mass_flow_laws():
    """Thrust enters as the product u Tmax:  Tmax dc/dTmax = sum_j u_j dc/du_j;  m' = -b Tmax u is
    linear in b:  b dc/db = the defect part of the mass rows."""
    w, P, x, wv = point("goddard_n1e3", 27, 13)
    Cd, beta, Tmax, b = w["params"]
    N, nx = w["N"], w["nx"]
    d = O.dpar_vjp_all(P, x, wv)
    Jtw = O.jtprod(P, x, wv)
    u = x[nx * (N + 1):nx * (N + 1) + N + 1]
    uterm = u @ Jtw[nx * (N + 1):nx * (N + 1) + N + 1]
    assert abs(Tmax * d[2] - uterm) <= 1e-12 * (abs(Tmax * d[2]) + np.abs(u * Jtw[nx * (N + 1):nx * (N + 1) + N + 1]).sum())
    c = O.evaluate(P, x, np.zeros(P.m), 1.0)["c"]
    X = x[:nx * (N + 1)].reshape(N + 1, nx)
    rows = [defect_row(P, w, 2, j) for j in range(N)]
    terms = [wv[r] * (c[r] - (X[j + 1, 2] - X[j, 2])) for j, r in enumerate(rows)]
    assert abs(b * d[3] - sum(terms)) <= 1e-12 * (abs(b * d[3]) + np.abs(terms).sum())
