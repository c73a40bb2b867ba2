"""Pins of the CPU oracle against facts fixed outside it (no GPU needed).

Each test checks the oracle against something other than itself: closed forms of the
paper's double-integrator example (Sec. 5), published constants of the Van der Pol limit
cycle, conservation laws of the cart-pole, discrete summation-by-parts of the heat
Laplacian, complex-step derivatives of the residual itself, brute-force structure
detection, and the adjoint identity.  A plausible slip anywhere in the oracle (a sign, a
dropped term, a wrong index or weight) fails at least one of these.
"""
import numpy as np
import pytest

from conftest import read_golden
from oracle import oracle as O
from paper_2510_03932_gb300 import synth

MODELS = ["vdp_n1e3", "cartpole_n1e5", "heat_n2e4", "dint", "quadrotor_n1e3", "goddard_n1e3",
          "vdp_n1e3:euler", "cartpole_n1e5:euler", "dint:euler", "quadrotor_n1e3:euler", "heat_n2e4:euler"]
# with path inequalities (counts are checked separately)
PATHED = ["vdp_n1e3+path", "cartpole_n1e5+path", "quadrotor_n1e3+path", "goddard_n1e3+path", "heat_n2e4+path",
          "vdp_n1e3:euler+path", "quadrotor_n1e3:euler+path"]


# with boundary inequalities b(X_0, X_N) <= 0 (trapezoidal scheme)
BINEQED = ["vdp_n1e3+bineq", "cartpole_n1e5+bineq", "dint+bineq", "quadrotor_n1e3+bineq", "goddard_n1e3+bineq",
           "heat_n2e4+bineq", "vdp_n1e3+path+bineq"]
# with the boundary cost g(X_0, X_N) added to the objective
BOLZAED = ["vdp_n1e3+bolza", "cartpole_n1e5+bolza", "dint+bolza", "quadrotor_n1e3+bolza", "goddard_n1e3+bolza",
           "heat_n2e4+bolza", "vdp_n1e3:euler+bolza", "dint:euler+path+bolza", "vdp_n1e3+bineq+bolza"]


def small(name, N):
    """A workload at horizon N; the suffix ":euler" selects the forward Euler scheme, "+path"
    attaches the model's path inequalities and "+bineq" its boundary inequalities."""
    name, *plus = name.split("+")
    base, _, scheme = name.partition(":")
    w = synth.with_horizon(synth.workload(base), N)
    if scheme:
        w["scheme"] = scheme
    if "path" in plus:
        w = synth.with_path(w)
    if "bineq" in plus:
        w = synth.with_bineq(w)
    if "bolza" in plus:
        w = synth.with_bolza(w)
    return w


def rand_point(w, rng):
    n, m = synth.dims(w)
    d = synth.DIST[w["dist"]]
    N1 = w["N"] + 1
    if "xc" in d:
        X = np.concatenate([rng.uniform(lo, hi, N1)[:, None] for lo, hi in d["xc"]], axis=1).ravel()
    else:
        X = rng.uniform(*d["x"], w["nx"] * N1)
    parts = [X, rng.uniform(*d["u"], w["nu"] * synth.control_nodes(w))]
    if w.get("free_tf"):
        parts.append(rng.uniform(*d["tf"], 1))
    return np.concatenate(parts), rng.standard_normal(m)


# ---------------------------------------------------------------------------------------
# Counts and structure
# ---------------------------------------------------------------------------------------
# per node: (J entries of one defect-row set, H entries of one node block)
NODE_COUNTS = {"vdp": (10, 4), "cartpole": (22, 7), "heat": (382, 65), "dint": (8, 1), "quadrotor": (68, 20),
               # Goddard: rows r {r, v | r, v | tf}, v {r, v, m | r, v, m | u | u | tf}, m {m | m | u | u | tf};
               # Hessian block (r,r) (v,r) (v,v) (m,r) (m,v) (m,m) (u,m) plus the tf row on r, v, m, u
               "goddard": (19, 11),
               # forward Euler: one node's side of each row plus the identity on X_{i+1,k}; the
               # Hessian blocks of the N nodes that carry a control
               "vdp:euler": (7, 4), "cartpole:euler": (15, 7), "dint:euler": (6, 1), "quadrotor:euler": (43, 20),
               "heat:euler": (255, 65)}


@pytest.mark.parametrize("name", MODELS)
@pytest.mark.parametrize("N", [1, 2, 7])
def test_counts_closed_form(name, N):
    w = small(name, N)
    P = O.Problem(w)
    nx, nu = w["nx"], w["nu"]
    nb = nx + synth.final_rows(w)
    euler = w.get("scheme") == "euler"
    jn, hn = NODE_COUNTS[w["model"] + (":euler" if euler else "")]
    nun = N if euler else N + 1
    assert P.n == nx * (N + 1) + nu * nun + (1 if w.get("free_tf") else 0)
    assert P.m == nb + nx * N
    assert P.nnzj == nb + jn * N
    assert P.nnzh == hn * nun


@pytest.mark.parametrize("name", MODELS)
def test_structure_sorted_unique(name):
    P = O.Problem(small(name, 5))
    for rows, cols, lower in [(*O.jac_structure(P), False), (*O.hess_structure(P), True)]:
        key = rows.astype(np.int64) * (1 << 32) + cols
        assert np.all(np.diff(key) > 0), "COO must be sorted by (row, col) without duplicates"
        if lower:
            assert np.all(rows >= cols)
        assert rows.min() >= 0 and cols.min() >= 0


def dense_jac_cs(P, x):
    cols = []
    for i in range(P.n):
        e = np.zeros(P.n); e[i] = 1.0
        cols.append(O.cs_cons(P, x, e))
    return np.array(cols).T  # m x n


def dense_hess_cs(P, x, y, sigma):
    cols = []
    for i in range(P.n):
        e = np.zeros(P.n); e[i] = 1.0
        cols.append(O.cs_lagrangian_grad(P, x, e, y, sigma))
    return np.array(cols).T  # n x n


@pytest.mark.parametrize("name", MODELS + PATHED + BINEQED + BOLZAED)
def test_structure_matches_bruteforce_detection(name):
    """An entry is structural iff it is nonzero at one of 8 random points (complex step)."""
    w = small(name, 2 if name.startswith("heat") else 3)
    P = O.Problem(w)
    rng = np.random.default_rng(7)
    jmask = np.zeros((P.m, P.n), bool)
    hmask = np.zeros((P.n, P.n), bool)
    for _ in range(8):
        x, y = rand_point(w, rng)
        jmask |= dense_jac_cs(P, x) != 0.0
        hmask |= np.tril(dense_hess_cs(P, x, y, 1.0)) != 0.0
    jr, jc = O.jac_structure(P)
    hr, hc = O.hess_structure(P)
    jm = np.zeros_like(jmask); jm[jr, jc] = True
    hm = np.zeros_like(hmask); hm[hr, hc] = True
    assert np.array_equal(jm, jmask)
    if w.get("bineq") or w.get("bolza"):
        # one Hessian template for every node: a boundary row's or the boundary cost's squared
        # term on component k puts (k, k) in every node's block; away from nodes 0 and N it is
        # an explicit zero
        nx = w["nx"]
        ba = np.array(w["bineq"]["a"]) if w.get("bineq") else np.zeros((0, 2 * nx))
        if w.get("bolza"):
            ba = np.vstack([ba, np.array(w["bolza"]["a"])[None, :]])
        sq = [k for k in range(nx) if np.any(ba[:, k] != 0) or np.any(ba[:, nx + k] != 0)]
        allowed = np.zeros_like(hm)
        for j in range(w["N"] + 1):
            for k in sq:
                allowed[nx * j + k, nx * j + k] = True
        assert not np.any(hmask & ~hm) and not np.any(hm & ~hmask & ~allowed)
    else:
        assert np.array_equal(hm, hmask)


# ---------------------------------------------------------------------------------------
# Derivative values against complex step of the residual / objective / Lagrangian gradient
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("name", MODELS + PATHED + BINEQED + BOLZAED)
def test_jacobian_gradient_hessian_vs_complex_step(name):
    w = small(name, 2 if name.startswith("heat") else 4)
    P = O.Problem(w)
    rng = np.random.default_rng(11)
    x, y = rand_point(w, rng)
    sigma = 0.7
    ev = O.evaluate(P, x, y, sigma)
    Jcs = dense_jac_cs(P, x)
    jr, jc = O.jac_structure(P)
    np.testing.assert_allclose(ev["jac"], Jcs[jr, jc], rtol=1e-13, atol=1e-15)
    gcs = np.array([O.cs_obj(P, x, np.eye(P.n)[i]) for i in range(P.n)])
    np.testing.assert_allclose(ev["g"], gcs, rtol=1e-13, atol=1e-15)
    Hcs = dense_hess_cs(P, x, y, sigma)
    hr, hc = O.hess_structure(P)
    np.testing.assert_allclose(ev["hess"], Hcs[hr, hc], rtol=1e-12, atol=1e-14)
    # the complex-step Hessian of an exact gradient is symmetric
    np.testing.assert_allclose(Hcs, Hcs.T, rtol=1e-12, atol=1e-12)
    # loose central finite differences as an independent sanity check of the residual
    hfd = 1e-6
    e = np.zeros(P.n); e[1] = 1.0
    cfd = (O.evaluate(P, x + hfd * e, y, sigma)["c"] - O.evaluate(P, x - hfd * e, y, sigma)["c"]) / (2 * hfd)
    np.testing.assert_allclose(cfd, Jcs[:, 1], rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("name", ["vdp_n1e3", "cartpole_n1e5", "heat_n2e4", "quadrotor_n1e3"])
def test_hessian_special_cases(name):
    """y = 0, sigma = 1: H is the weighted cost Hessian 2 w_j diag(q, r).
    sigma = 0, y = e_r: H is the Hessian of the single defect r (supported on 2 nodes)."""
    w = small(name, 3)
    P = O.Problem(w)
    rng = np.random.default_rng(3)
    x, _ = rand_point(w, rng)
    hr, hc = O.hess_structure(P)
    h = w["T"] / w["N"]
    ev = O.evaluate(P, x, np.zeros(P.m), 1.0)
    nx, nu, N = w["nx"], w["nu"], w["N"]
    diag = np.concatenate([np.tile(2.0 * np.array(w["q"]), N + 1), np.tile(2.0 * np.array(w["r"]), N + 1)])
    wts = np.concatenate([np.repeat([h / 2] + [h] * (N - 1) + [h / 2], nx),
                          np.repeat([h / 2] + [h] * (N - 1) + [h / 2], nu)])
    expect = np.where(hr == hc, (diag * wts)[hr], 0.0)
    np.testing.assert_allclose(ev["hess"], expect, rtol=1e-15, atol=0)
    r = P.m - 1  # last defect of the last component: nodes N-1 and N
    y = np.zeros(P.m); y[r] = 1.0
    ev = O.evaluate(P, x, y, 0.0)
    Hcs = dense_hess_cs(P, x, y, 0.0)
    np.testing.assert_allclose(ev["hess"], Hcs[hr, hc], rtol=1e-12, atol=1e-14)
    nz = ev["hess"] != 0
    node_of = lambda v: np.where(v < nx * (N + 1), v // nx, (v - nx * (N + 1)) // nu)
    assert set(np.unique(node_of(hr[nz]))) <= {N - 1, N}


# ---------------------------------------------------------------------------------------
# Closed form: the paper's double integrator (Sec. 5)
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("N", [10, 100, 1000])
def test_dint_closed_form(N):
    gd = read_golden("dint_double_integrator.txt")
    w = small("dint", N)
    P = O.Problem(w)
    h = 1.0 / N
    t = np.arange(N + 1) * h
    x1 = gd["x1_coef0"] + gd["x1_coef2"] * t**2 + gd["x1_coef3"] * t**3
    x2 = gd["x2_coef1"] * t + gd["x2_coef2"] * t**2
    u = gd["u_coef0"] + gd["u_coef1"] * t
    X = np.stack([x1, x2], 1).ravel()
    x = np.concatenate([X, u])
    y = np.random.default_rng(0).standard_normal(P.m)
    ev = O.evaluate(P, x, y, 1.0)
    c = ev["c"]
    # boundary rows are the state values themselves (bit-exact)
    assert c[0] == X[0] and c[1] == X[1] and c[2] == X[2 * N] and c[3] == X[2 * N + 1]
    np.testing.assert_allclose(c[4:4 + N], gd["defect1_h3_coef"] * h**3, rtol=1e-6, atol=4e-16)
    np.testing.assert_allclose(c[4 + N:], gd["defect2"], atol=4e-15)
    assert abs(ev["f"] - (gd["optimal_cost"] + gd["cost_h2_coef"] * h**2)) < 1e-13
    # the Jacobian is constant: +-1 and -h/2, bit-exact
    jr, jc = O.jac_structure(P)
    J = ev["jac"]
    assert set(np.unique(J)) <= {1.0, -1.0, -h / 2}
    Jd = np.zeros((P.m, P.n)); Jd[jr, jc] = J
    for j in range(N):
        r1, r2 = 4 + j, 4 + N + j
        assert Jd[r1, 2 * j] == -1 and Jd[r1, 2 * j + 2] == 1
        assert Jd[r1, 2 * j + 1] == -h / 2 and Jd[r1, 2 * j + 3] == -h / 2
        assert Jd[r2, 2 * j + 1] == -1 and Jd[r2, 2 * j + 3] == 1
        uj = 2 * (N + 1) + j
        assert Jd[r2, uj] == -h / 2 and Jd[r2, uj + 1] == -h / 2
    # H is diagonal on u with value sigma * w_j (d2 (u^2/2) = 1)
    hr, hc = O.hess_structure(P)
    assert np.all(hr == hc) and np.all(hr >= 2 * (N + 1))
    wts = np.array([h / 2] + [h] * (N - 1) + [h / 2])
    assert np.array_equal(ev["hess"], wts)


# ---------------------------------------------------------------------------------------
# Physics pins of the model right-hand sides
# ---------------------------------------------------------------------------------------
def test_vdp_limit_cycle_period_and_amplitude():
    """Integrate u = 0 with the oracle's own trapezoidal defect (Newton on c_{.,0} = 0 at N=1)
    and recover the published period and amplitude of the mu = 1 limit cycle."""
    gd = read_golden("vdp_limit_cycle.txt")
    hstep = 0.004
    w = dict(synth.workload("vdp_n1e3"), N=1, T=hstep, params=[gd["mu"]])
    P = O.Problem(w)
    jr, jc = O.jac_structure(P)
    X = np.array([2.0, 0.0])
    traj = [X.copy()]
    for _ in range(int(40.0 / hstep)):
        Xn = X.copy()
        for _ in range(8):
            x = np.concatenate([X, Xn, [0.0, 0.0]])
            ev = O.evaluate(P, x, np.zeros(P.m), 1.0)
            Jd = np.zeros((P.m, P.n)); Jd[jr, jc] = ev["jac"]
            res = ev["c"][2:4]
            dX = np.linalg.solve(Jd[2:4, 2:4], -res)
            Xn = Xn + dX
            if np.max(np.abs(dX)) < 1e-15:
                break
        X = Xn
        traj.append(X.copy())
    traj = np.array(traj)
    t = np.arange(len(traj)) * hstep
    x1 = traj[:, 0]
    up = np.where((x1[:-1] < 0) & (x1[1:] >= 0))[0]
    tc = t[up] + hstep * (-x1[up]) / (x1[up + 1] - x1[up])
    period = np.mean(np.diff(tc[-3:]))
    amp = np.max(np.abs(x1[t > 20.0]))
    assert abs(period - gd["period"]) < 2e-3 * gd["period"]
    assert abs(amp - gd["amplitude"]) < 2e-3 * gd["amplitude"]


def test_cartpole_conservation_laws():
    """With F the horizontal force on the cart: d/dt of the horizontal momentum
    (mc+mp) pd + mp l w cos(th) equals F, and d/dt of the energy
    1/2 (mc+mp) pd^2 + mp l pd w cos(th) + 1/2 mp l^2 w^2 - mp g l cos(th) equals F pd.
    The two identities fix both accelerations."""
    w = synth.workload("cartpole_n1e5")
    P = O.Problem(small("cartpole_n1e5", 1))
    mc, mp, l, g = w["params"]
    rng = np.random.default_rng(5)
    for _ in range(50):
        p, pd, th, om, F = rng.uniform(-3, 3, 5)
        f = O.model_f(P, [p, pd, th, om, F])
        assert f[0] == pd and f[2] == om
        pdd, thdd = f[1], f[3]
        dmom = (mc + mp) * pdd + mp * l * (thdd * np.cos(th) - om**2 * np.sin(th))
        dE = ((mc + mp) * pd * pdd + mp * l * (pdd * om * np.cos(th) + pd * thdd * np.cos(th)
                                               - pd * om**2 * np.sin(th))
              + mp * l**2 * om * thdd + mp * g * l * np.sin(th) * om)
        assert abs(dmom - F) < 1e-12 * (1 + abs(F) + abs(pdd) + abs(thdd))
        assert abs(dE - F * pd) < 1e-12 * (1 + abs(F * pd) + abs(pdd) + abs(thdd)) * 10


def test_heat_laplacian_boundary_conditions():
    """Sum of the discrete Laplacian telescopes to (x_0 - x_1) + (x_{n+1} - x_n) over dx^2:
    with the Dirichlet ghost x_0 = u and the Neumann ghost x_{n+1} = x_n this is
    (u - x_1) / dx^2.  A constant profile equal to u has zero Laplacian everywhere, and a
    linear profile has zero second difference away from the Neumann end."""
    P = O.Problem(small("heat_n2e4", 1))
    n = 64
    dx = 1.0 / n
    rng = np.random.default_rng(9)
    for _ in range(10):
        xc = rng.uniform(0, 1, n); u = rng.uniform(-1, 1)
        f = O.model_f(P, np.concatenate([xc, [u]]))
        lap = f + xc**3
        assert abs(lap.sum() - (u - xc[0]) / dx**2) < 1e-9 * np.abs(lap).sum()
    cval = 0.37
    f = O.model_f(P, np.full(n + 1, cval))
    np.testing.assert_allclose(f, -cval**3, rtol=1e-13)
    a, b = 0.2, 0.01
    xc = a + b * np.arange(1, n + 1)
    f = O.model_f(P, np.concatenate([xc, [a]]))
    np.testing.assert_allclose(f[:-1], -xc[:-1] ** 3, rtol=1e-9, atol=1e-9)
    assert abs(f[-1] - (-b / dx**2 - xc[-1] ** 3)) < 1e-9


def test_quadrotor_hover_and_small_angle_linearisation():
    """Hover (level attitude, thrust u1 = g, no rates) is an equilibrium: every defect is
    exactly zero.  At level attitude (x7 = x8 = x9 = 0) the Jacobian is the small-angle model
    of the rigid body, written out by hand below: the thrust tilts into x2' and x4', and the
    angle rates are the inputs u2, u3, u4 with first-order couplings through x7 and x8."""
    w = small("quadrotor_n1e3", 1)
    P = O.Problem(w)
    g = w["params"][0]
    N, nx, nu = 1, 9, 4
    X = np.zeros(nx * (N + 1))
    U = np.tile([g, 0.0, 0.0, 0.0], N + 1)
    ev = O.evaluate(P, np.concatenate([X, U]), np.zeros(P.m), 1.0)
    assert np.all(ev["c"][nx:] == 0.0)
    # linearisation at x7 = x8 = x9 = 0 with arbitrary controls (exact values at zero angles)
    rng = np.random.default_rng(21)
    u1, u2, u3, u4 = rng.uniform(-5, 5, 4)
    z = np.zeros(13)
    z[:6] = rng.uniform(-1, 1, 6)
    z[9:] = [u1, u2, u3, u4]
    x = np.concatenate([z[:9], z[:9], z[9:], z[9:]])
    ev = O.evaluate(P, x, np.zeros(P.m), 1.0)
    jr, jc = O.jac_structure(P)
    Jd = np.zeros((P.m, P.n)); Jd[jr, jc] = ev["jac"]
    h = w["T"] / N
    # d f_k / d z_v at level attitude (rows: f1..f9, columns: x1..x9, u1..u4)
    A = np.zeros((9, 13))
    A[0, 1] = A[2, 3] = A[4, 5] = 1.0                  # position derivatives are velocities
    A[1, 7] = u1                                       # x2' = u1 sin(x8) ~ u1 x8
    A[3, 6] = -u1                                      # x4' = -u1 sin(x7) ~ -u1 x7
    A[5, 9] = 1.0                                      # x6' = u1 - g
    A[6, 6], A[6, 10] = u3, 1.0                        # x7' = u2 + u3 x7
    A[7, 6], A[7, 11] = -u2, 1.0                       # x8' = u3 - u2 x7
    A[8, 7], A[8, 12] = u2, 1.0                        # x9' = u2 x8 + u4
    cols0 = [k for k in range(9)] + [9 * (N + 1) + i for i in range(4)]
    cols1 = [9 + k for k in range(9)] + [9 * (N + 1) + 4 + i for i in range(4)]
    rows = nx + np.arange(9) * N
    expect0 = -h / 2 * A - np.hstack([np.eye(9), np.zeros((9, 4))])
    expect1 = -h / 2 * A + np.hstack([np.eye(9), np.zeros((9, 4))])
    np.testing.assert_allclose(Jd[np.ix_(rows, cols0)], expect0, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(Jd[np.ix_(rows, cols1)], expect1, rtol=1e-14, atol=1e-15)


def test_quadrotor_rotation_invariants():
    """The thrust acts along the body axis: (x2', x4', x6' + g) = u1 R e3 with R a rotation,
    so its norm is |u1| for every attitude.  The angle rates rotate (u2, u3) by x7:
    (x7' cos x8)^2 + x8'^2 = u2^2 + u3^2, and x9' - u4 = x7' sin x8."""
    w = small("quadrotor_n1e3", 1)
    P = O.Problem(w)
    g = w["params"][0]
    rng = np.random.default_rng(23)
    for _ in range(50):
        z = rng.uniform(-1.2, 1.2, 13)
        z[9:] = rng.uniform(-8, 8, 4)
        f = O.model_f(P, z)
        assert f[0] == z[1] and f[2] == z[3] and f[4] == z[5]
        thrust = np.sqrt(f[1] ** 2 + f[3] ** 2 + (f[5] + g) ** 2)
        assert abs(thrust - abs(z[9])) < 1e-13 * (1 + abs(z[9]))
        assert abs((f[6] * np.cos(z[7])) ** 2 + f[7] ** 2 - (z[10] ** 2 + z[11] ** 2)) < 1e-12 * (1 + z[10] ** 2 + z[11] ** 2)
        assert abs((f[8] - z[12]) - f[6] * np.sin(z[7])) < 1e-12 * (1 + abs(f[6]))


@pytest.mark.parametrize("N", [5, 16, 1000])
def test_quadrotor_tracking_cost_closed_form(N):
    """With every state and control at zero the running cost is the reference alone:
    1/2 [sin^2(2 pi t) + 4 sin^2(4 pi t) + 4 t^2] on [0, 1].  The trapezoidal rule integrates
    cos(2 pi k t) exactly to zero over a period when N does not divide k, and has the error
    h^2/12 (f'(1) - f'(0)) on t^2, so F = 1/2 (1/2 + 2 + 4/3 + 2 h^2/3) = 23/12 + h^2/3."""
    w = small("quadrotor_n1e3", N)
    P = O.Problem(w)
    h = 1.0 / N
    ev = O.evaluate(P, np.zeros(P.n), np.zeros(P.m), 1.0)
    assert abs(ev["f"] - (23.0 / 12.0 + h * h / 3.0)) < 1e-14 * 2
    # on the reference the tracked gradient entries vanish (up to the rounding of sin)
    t = np.arange(N + 1) * h
    X = np.zeros((N + 1, 9))
    X[:, 0], X[:, 2], X[:, 4] = np.sin(2 * np.pi * t), 2 * np.sin(4 * np.pi * t), 2 * t
    ev = O.evaluate(P, np.concatenate([X.ravel(), np.zeros(4 * (N + 1))]), np.zeros(P.m), 1.0)
    assert np.max(np.abs(ev["g"])) < 1e-15 and abs(ev["f"]) < 1e-30


def test_goddard_gravity_and_energy_balance():
    """Without speed the only acceleration is the inverse-square gravity -1/r^2 (normalised
    units) plus thrust; along any state the specific energy e = v^2/2 - 1/r changes at the
    rate of thrust power minus drag power per unit mass: de/dt = v (u Tmax - Cd v^2 exp(-beta
    (r - 1))) / m.  The mass flow is -b Tmax u.  Together these fix every term of v'."""
    w = small("goddard_n1e3", 1)
    P = O.Problem(w)
    Cd, beta, Tmax, b = w["params"]
    rng = np.random.default_rng(29)
    for _ in range(50):
        r, v, m, u = rng.uniform(1.0, 1.03), rng.uniform(-0.2, 0.2), rng.uniform(0.5, 1.0), rng.uniform(0, 1)
        f = O.model_f(P, [r, 0.0, m, u])
        assert abs(f[1] - (u * Tmax / m - 1.0 / r**2)) < 1e-15 * 8
        f = O.model_f(P, [r, v, m, u])
        assert f[0] == v and f[2] == -b * Tmax * u
        de = v * f[1] + f[0] / r**2
        expect = v * (u * Tmax - Cd * v * v * np.exp(-beta * (r - 1.0))) / m
        assert abs(de - expect) < 1e-13 * (1 + abs(v) * (u * Tmax + Cd * v * v) / m)


def test_free_final_time_reduces_to_fixed_horizon():
    """With tf appended to x and set to T, the residual, the Jacobian entries on X and U, the
    node Hessian blocks and the objective equal those of the fixed-horizon transcription (which
    the other pins fix); the Lagrange cost is linear in tf, so dF/dtf tf = F."""
    wf = dict(small("vdp_n1e3", 7), T=2.5)
    wt = dict(wf, free_tf=True, T=1.0)
    Pf, Pt = O.Problem(wf), O.Problem(wt)
    assert Pt.n == Pf.n + 1 and Pt.m == Pf.m
    rng = np.random.default_rng(31)
    x, y = rand_point(wf, rng)
    xt = np.concatenate([x, [2.5]])
    ef, et = O.evaluate(Pf, x, y, 0.8), O.evaluate(Pt, xt, y, 0.8)
    np.testing.assert_allclose(et["c"], ef["c"], rtol=1e-15, atol=1e-16)
    assert abs(et["f"] - ef["f"]) <= 1e-15 * abs(ef["f"])
    np.testing.assert_allclose(et["g"][:-1], ef["g"], rtol=1e-15, atol=1e-16)
    assert abs(et["g"][-1] * 2.5 - ef["f"]) <= 1e-13 * abs(ef["f"])
    jr, jc = O.jac_structure(Pt)
    keep = jc != Pt.n - 1
    np.testing.assert_allclose(et["jac"][keep], ef["jac"], rtol=1e-15, atol=1e-16)
    hr, hc = O.hess_structure(Pt)
    keep = hr != Pt.n - 1
    np.testing.assert_allclose(et["hess"][keep], ef["hess"], rtol=1e-15, atol=1e-16)


def test_goddard_mayer_objective_and_final_row():
    """max r(tf) is the linear terminal cost F = -r_N: gradient -1 on r_N and nothing else
    (no running cost, so dF/dtf = 0 and the Hessian has no cost entries); the single final row
    is m_N with a unit Jacobian entry."""
    w = small("goddard_n1e3", 6)
    P = O.Problem(w)
    rng = np.random.default_rng(37)
    x, y = rand_point(w, rng)
    ev = O.evaluate(P, x, np.zeros(P.m), 1.0)
    rN = 3 * 6
    assert ev["f"] == -x[rN]
    g = np.zeros(P.n); g[rN] = -1.0
    assert np.array_equal(ev["g"], g)
    assert np.all(ev["hess"] == 0.0)
    assert ev["c"][3] == x[3 * 6 + 2]
    jr, jc = O.jac_structure(P)
    assert jr[3] == 3 and jc[3] == 3 * 6 + 2 and ev["jac"][3] == 1.0


@pytest.mark.parametrize("N", [10, 100, 1000])
def test_euler_local_error_and_rectangle_cost_closed_forms(N):
    """Forward Euler on the double integrator (paper Sec. 3 scheme).  At the exact solution of
    x1' = x2, x2' = u with u = 1, x(0) = 0 (x1 = t^2/2, x2 = t) the defects are the local
    truncation errors h^2 x1''/2 = h^2/2 and 0.  The rectangle rule of 1/2 u^2 with
    u_i = a + b t_i (left end points) sums to h/2 [N a^2 + a b h N (N-1) + b^2 h^2 (N-1) N (2N-1) / 6]."""
    w = small("dint:euler", N)
    P = O.Problem(w)
    h = 1.0 / N
    t = np.arange(N + 1) * h
    X = np.stack([t**2 / 2, t], 1).ravel()
    x = np.concatenate([X, np.ones(N)])
    ev = O.evaluate(P, x, np.zeros(P.m), 1.0)
    nb = 4
    np.testing.assert_allclose(ev["c"][nb:nb + N], h * h / 2, rtol=1e-9, atol=1e-16)
    np.testing.assert_allclose(ev["c"][nb + N:], 0.0, atol=1e-15)
    a, b = 0.7, -1.3
    x = np.concatenate([X, a + b * t[:N]])
    F = O.evaluate(P, x, np.zeros(P.m), 1.0)["f"]
    expect = h / 2 * (N * a * a + a * b * h * N * (N - 1) + b * b * h * h * (N - 1) * N * (2 * N - 1) / 6)
    assert abs(F - expect) < 1e-13 * abs(expect)
    # the Jacobian of the linear dynamics: -1 / +1 identities and -h couplings, no U_N column
    jr, jc = O.jac_structure(P)
    assert set(np.unique(ev["jac"])) <= {1.0, -1.0, -h}
    assert jc.max() < P.n and P.n == 2 * (N + 1) + N


def test_euler_vdp_mu_derivative_vs_complex_step():
    w = small("vdp_n1e3:euler", 13)
    P = O.Problem(w, mu=1.4)
    rng = np.random.default_rng(43)
    x, _ = rand_point(w, rng)
    wv = rng.standard_normal(P.m)
    got = O.dpar_vjp(P, x, wv)
    ref = wv @ O.cs_cons(P, x, np.zeros(P.n), dmu=1.0)
    assert abs(got - ref) <= 1e-13 * (1 + abs(ref))


@pytest.mark.parametrize("name", PATHED)
def test_path_rows_counts_and_boundary_points(name):
    """Path inequalities add one row per inequality and controlled node after the defects, with
    one Jacobian entry per variable in the row's support and Hessian diagonals for its squared
    terms.  On their boundary the rows vanish: x2 = -0.4 for the Van der Pol half-space, points
    (2 cos phi, sin phi) of the cart-pole ellipse, points of the quadrotor's keep-out circle."""
    w = small(name, 6)
    wp = {k: v for k, v in w.items() if k != "path"}
    P, P0 = O.Problem(w), O.Problem(wp)
    nun = synth.control_nodes(w)
    pa = np.array(w["path"]["a"]); pl = np.array(w["path"]["l"])
    supp = (pa != 0) | (pl != 0)
    assert P.n == P0.n and P.m == P0.m + len(w["path"]["r"]) * nun
    assert P.nnzj == P0.nnzj + int(supp.sum()) * nun
    hr0, hc0 = O.hess_structure(P0)
    hr, hc = O.hess_structure(P)
    assert set(zip(hr0, hc0)) <= set(zip(hr, hc))
    rng = np.random.default_rng(47)
    x, _ = rand_point(w, rng)
    nx, N = w["nx"], w["N"]
    uoff = nx * (N + 1)
    base = P.m - len(w["path"]["r"]) * nun
    if w["model"] == "vdp":
        x[1::2][:N + 1] = -0.4  # x2 at every node
        c = O.evaluate(P, x, np.zeros(P.m), 1.0)["c"]
        assert np.all(c[base:base + nun] == 0.0)
    if w["model"] == "cartpole":
        phi = rng.uniform(0, 2 * np.pi, N + 1)
        x[0:uoff:4] = 2 * np.cos(phi); x[2:uoff:4] = np.sin(phi)
        c = O.evaluate(P, x, np.zeros(P.m), 1.0)["c"]
        np.testing.assert_allclose(c[base:base + nun], 0.0, atol=4e-16)
    if w["model"] == "quadrotor":
        phi = rng.uniform(0, 2 * np.pi, N + 1)
        x[0:uoff:9] = 0.5 + 0.2 * np.cos(phi); x[2:uoff:9] = 0.5 + 0.2 * np.sin(phi)
        c = O.evaluate(P, x, np.zeros(P.m), 1.0)["c"]
        np.testing.assert_allclose(c[base + nun:base + 2 * nun], 0.0, atol=4e-16)


@pytest.mark.parametrize("name", BINEQED)
def test_boundary_inequalities_counts_and_boundary_points(name):
    """Boundary inequalities add one row each after every other row, one Jacobian entry per
    variable of (X_0, X_N) in the row's support, and a (k, k) entry in every node's Hessian
    block for a squared term on component k (values non-zero only at nodes 0 and N).  On their
    boundary the rows vanish: the Van der Pol terminal circle |X_N| = 1/2, the cart-pole's
    upright pole X_{N,3} = pi +- 0.1; a linear row's Jacobian entries are its constant
    coefficients."""
    w = small(name, 5)
    wb = {k: v for k, v in w.items() if k != "bineq"}
    P, P0 = O.Problem(w), O.Problem(wb)
    nx, N = w["nx"], w["N"]
    ba, bl = np.array(w["bineq"]["a"]), np.array(w["bineq"]["l"])
    nbin = len(w["bineq"]["r"])
    assert P.n == P0.n and P.m == P0.m + nbin
    assert P.nnzj == P0.nnzj + int(((ba != 0) | (bl != 0)).sum())
    hr0, hc0 = O.hess_structure(P0)
    hr, hc = O.hess_structure(P)
    assert set(zip(hr0, hc0)) <= set(zip(hr, hc))
    sq = sorted({k for q in range(nbin) for k in range(nx) if ba[q, k] != 0 or ba[q, nx + k] != 0})
    new = set(zip(hr, hc)) - set(zip(hr0, hc0))
    assert new == {(nx * j + k, nx * j + k) for j in range(N + 1) for k in sq
                   if (nx * j + k, nx * j + k) not in set(zip(hr0, hc0))}
    rng = np.random.default_rng(53)
    x, y = rand_point(w, rng)
    # with only the boundary multipliers non-zero, H is zero away from nodes 0 and N
    yb = np.zeros(P.m); yb[P.m - nbin:] = y[P.m - nbin:]
    ev = O.evaluate(P, x, yb, 0.0)
    mid = (hr >= nx) & (hr < nx * N)
    assert np.all(ev["hess"][mid] == 0.0)
    jr, jc = O.jac_structure(P)
    if w["model"] == "vdp":
        phi = rng.uniform(0, 2 * np.pi)
        x[2 * N] = 0.5 * np.cos(phi); x[2 * N + 1] = 0.5 * np.sin(phi)
        ev = O.evaluate(P, x, y, 1.0)
        r0 = P.m - nbin
        assert abs(ev["c"][r0]) <= 4e-16
        lin = jr == r0 + 1   # X_{N,1} - X_{0,1} - 1: entries -1 on X_{0,1}, +1 on X_{N,1}
        assert list(jc[lin]) == [0, 2 * N] and list(ev["jac"][lin]) == [-1.0, 1.0]
        assert ev["c"][r0 + 1] == (x[2 * N] - x[0]) - 1.0
    if w["model"] == "cartpole":
        for th in (np.pi + 0.1, np.pi - 0.1):
            x[4 * N + 2] = th
            assert abs(O.evaluate(P, x, y, 1.0)["c"][P.m - nbin]) <= 4e-16


@pytest.mark.parametrize("name", ["vdp_n1e3", "quadrotor_n1e3", "goddard_n1e3", "heat_n2e4"])
def test_boundary_cost_at_its_target_and_counts(name):
    """The boundary cost adds no row and no Jacobian entry, and its (k, k) template diagonals;
    at z = b with l = 0 it adds nothing to F and to the gradient (the penalty's minimum), and a
    step delta along X_{N,k} adds a_k delta^2 (+ l delta for a linear term) to F."""
    w = small(name, 6)
    nx, N = w["nx"], w["N"]
    wq = synth.with_bolza(w)
    lin = [0.0] * (2 * nx)
    wq = dict(wq, bolza=dict(wq["bolza"], l=lin, a=[0.0] * nx + wq["bolza"]["a"][nx:]))
    P, P0 = O.Problem(wq), O.Problem(w)
    assert (P.n, P.m, P.nnzj) == (P0.n, P0.m, P0.nnzj) and P.nnzh >= P0.nnzh
    rng = np.random.default_rng(61)
    x, y = rand_point(w, rng)
    bN = np.array(wq["bolza"]["b"][nx:])
    x[nx * N:nx * N + nx] = bN
    e1, e0 = O.evaluate(P, x, y, 1.0), O.evaluate(P0, x, y, 1.0)
    assert e1["f"] == e0["f"]
    assert np.array_equal(e1["g"], e0["g"])
    for k in range(nx):
        xd = x.copy(); xd[nx * N + k] += 0.125
        df = O.evaluate(P, xd, y, 1.0)["f"] - O.evaluate(P0, xd, y, 1.0)["f"]
        assert abs(df - 1.5 * 0.125 ** 2) <= 1e-13 * (1 + abs(e0["f"]))


def test_boundary_cost_refused_with_euler_on_the_last_state():
    w = small("vdp_n1e3:euler", 5)
    wb = synth.with_bolza(w)
    O.Problem(wb)   # linear X_N terms are accepted
    a = list(wb["bolza"]["a"]); a[-1] = 1.0
    with pytest.raises(ValueError):
        O.Problem(dict(wb, bolza=dict(wb["bolza"], a=a)))


def test_boundary_inequalities_refused_with_euler():
    w = synth.with_bineq(small("vdp_n1e3:euler", 5))
    with pytest.raises(ValueError):
        O.Problem(w)


# ---------------------------------------------------------------------------------------
# Products and the parameter derivative
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("name", MODELS + PATHED + BINEQED + BOLZAED)
def test_products_vs_complex_step_and_adjoint(name):
    w = small(name, 3 if name.startswith("heat") else 9)
    P = O.Problem(w)
    rng = np.random.default_rng(13)
    x, y = rand_point(w, rng)
    v = rng.uniform(-1, 1, P.n)
    wv = rng.standard_normal(P.m)
    sigma = 1.3
    Jv = O.jprod(P, x, v)
    np.testing.assert_allclose(Jv, O.cs_cons(P, x, v), rtol=1e-13, atol=1e-14)
    Jtw = O.jtprod(P, x, wv)
    Jtw_cs = np.array([wv @ O.cs_cons(P, x, np.eye(P.n)[i]) for i in range(P.n)])
    np.testing.assert_allclose(Jtw, Jtw_cs, rtol=1e-12, atol=1e-13)
    assert abs(wv @ Jv - Jtw @ v) <= 1e-13 * (np.abs(wv) @ np.abs(Jv) + np.abs(Jtw) @ np.abs(v))
    Hv = O.hprod(P, x, y, sigma, v)
    np.testing.assert_allclose(Hv, O.cs_lagrangian_grad(P, x, v, y, sigma), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("name", MODELS + PATHED + BINEQED + BOLZAED)
def test_kkt_assembly_structure_and_action(name):
    """The KKT matrix [H + D, J^T; J, -delta_c I] (lower triangle): sorted, every diagonal
    present once, nnz = nnz_H + nnz_J + m + (diagonals H lacks); its symmetric action on
    (v, w) is (H v + D v + J^T w, J v - delta_c w) with the oracle's own products."""
    w = small(name, 3 if name.startswith("heat") else 7)
    P = O.Problem(w)
    rng = np.random.default_rng(41)
    x, y = rand_point(w, rng)
    sx = rng.uniform(0.1, 2.0, P.n)
    dw, dc = 1e-3, 1e-4
    rows, cols, vals = O.kkt(P, x, y, 0.9, sx, dw, dc)
    n, m = P.n, P.m
    key = rows.astype(np.int64) * (1 << 32) + cols
    assert np.all(np.diff(key) > 0) and np.all(rows >= cols)
    diag = rows == cols
    assert np.array_equal(np.sort(rows[diag]), np.arange(n + m))
    hr, hc = O.hess_structure(P)
    assert rows.size == P.nnzh + P.nnzj + m + (n - np.count_nonzero(hr == hc))
    v, wv = rng.standard_normal(n), rng.standard_normal(m)
    z = np.concatenate([v, wv])
    Kz = np.zeros(n + m)
    np.add.at(Kz, rows, vals * z[cols])
    off = ~diag
    np.add.at(Kz, cols[off], vals[off] * z[rows[off]])
    top = O.hprod(P, x, y, 0.9, v) + (sx + dw) * v + O.jtprod(P, x, wv)
    bot = O.jprod(P, x, v) - dc * wv
    np.testing.assert_allclose(Kz, np.concatenate([top, bot]), rtol=1e-12, atol=1e-12)


def test_dpar_vjp_vs_complex_step():
    w = small("vdp_n1e3", 17)
    P = O.Problem(w, mu=1.7)
    rng = np.random.default_rng(17)
    x, _ = rand_point(w, rng)
    wv = rng.standard_normal(P.m)
    got = O.dpar_vjp(P, x, wv)
    ref = wv @ O.cs_cons(P, x, np.zeros(P.n), dmu=1.0)
    assert abs(got - ref) <= 1e-13 * (1 + abs(ref))
    # the mixed derivative d/dmu (J^T w) is the gradient of (dc/dmu)^T w in x
    mixed = O.cs_jtprod_dmu(P, x, wv)
    fd = np.array([(O.dpar_vjp(P, x + 1e-6 * e, wv) - O.dpar_vjp(P, x - 1e-6 * e, wv)) / 2e-6
                   for e in np.eye(P.n)])
    np.testing.assert_allclose(mixed, fd, rtol=1e-6, atol=1e-8)


def test_shadow_bounds_value():
    w = small("cartpole_n1e5", 6)
    P = O.Problem(w)
    rng = np.random.default_rng(19)
    x, y = rand_point(w, rng)
    ev = O.evaluate(P, x, y, 1.0, shadow=True)
    for k in ["c", "g", "jac", "hess"]:
        mag, v = ev[k + "_mag"], np.abs(ev[k])
        # an output copied from an input is exact (bound 0); every computed one is bounded by
        # at least its own magnitude (the rounding of its last operation)
        assert np.all((mag == 0) | (mag >= v * (1 - 1e-15)))
    assert np.all(ev["c_mag"][:4] == 0)
    assert ev["f_mag"] >= abs(ev["f"])


def test_full_size_oracle_runs():
    """The oracle evaluates the N=1000 Van der Pol workload end to end on seeded inputs."""
    w = synth.workload("vdp_n1e3")
    P = O.Problem(w)
    d = synth.draw(w)
    ev = O.evaluate(P, d["x"], d["y"], w["sigma"])
    assert np.isfinite(ev["f"]) and ev["jac"].size == P.nnzj and ev["hess"].size == P.nnzh
    assert ev["c"][0] == d["x"][0] and ev["c"][1] == d["x"][1]
