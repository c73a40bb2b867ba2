"""Seeded synthetic inputs shared byte-for-byte by the CUDA path and the CPU oracle.

This module holds no arithmetic of the transcription method: it only draws numbers.
Generator: splitmix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014).  Element i of a stream with seed s is
mix(s + (i+1) * 0x9E3779B97F4A7C15); a uniform in [0,1) is the top 53 bits times 2^-53;
a standard normal is Box-Muller on two consecutive uniforms (the cosine branch).

Draw order for one problem instance, all from one stream: X (vector order), U, y, then
the product directions vn (length n) and vm (length m).
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class Stream:
    """A splitmix64 stream; `take(k)` returns the next k raw 64-bit outputs."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.pos = 0

    def take(self, k: int) -> np.ndarray:
        idx = np.arange(self.pos + 1, self.pos + 1 + k, dtype=np.uint64)
        self.pos += k
        with np.errstate(over="ignore"):
            z = self.seed + idx * _GAMMA
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, k: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.take(k) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        return lo + (hi - lo) * u

    def normal(self, k: int) -> np.ndarray:
        u = self.uniform(2 * k)
        u1, u2 = u[0::2], u[1::2]
        return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)

    def integers(self, k: int, lo: int, hi: int) -> np.ndarray:
        """Uniform integers in [lo, hi] (inclusive)."""
        u = self.uniform(k)
        return (lo + np.floor(u * (hi - lo + 1))).astype(np.int64)


# Value distributions of the five workloads (uniform bounds for X and U).
DIST = {
    "vdp": dict(x=(-1.0, 1.0), u=(-1.0, 1.0)),
    "cartpole": dict(x=(-1.0, 1.0), u=(-10.0, 10.0)),
    "heat": dict(x=(0.0, 1.0), u=(-1.0, 1.0)),
    "dint": dict(x=(-1.0, 1.0), u=(-1.0, 1.0)),
    "quadrotor": dict(x=(-1.0, 1.0), u=(-10.0, 10.0)),
    # Goddard: per-component ranges around the flight envelope (altitude r >= 1 with the drag
    # factor exp(-500 (r - 1)) finite, speed in [0, vmax], mass between the final and initial
    # mass), normalised thrust in [0, 1], free final time near the known optimum (~0.2)
    "goddard": dict(xc=[(1.0, 1.02), (0.0, 0.1), (0.6, 1.0)], u=(0.0, 1.0), tf=(0.15, 0.25)),
}


def draw_instance(seed: int, kind: str, nx: int, nu: int, N: int, m: int,
                  stream: Stream | None = None, free_tf: bool = False, unodes: int | None = None) -> dict:
    """x = [X (node-major, nx per node); U (nu per node) (; tf)], y ~ N(0,1), vn ~ U(-1,1),
    vm ~ N(0,1).  X is uniform on one range, or on a range per state component ("xc")."""
    s = stream if stream is not None else Stream(seed)
    d = DIST[kind]
    if "xc" in d:
        lo = np.array([r[0] for r in d["xc"]])
        hi = np.array([r[1] for r in d["xc"]])
        X = (lo + (hi - lo) * s.uniform(nx * (N + 1)).reshape(N + 1, nx)).ravel()
    else:
        X = s.uniform(nx * (N + 1), *d["x"])
    U = s.uniform(nu * ((N + 1) if unodes is None else unodes), *d["u"])
    parts = [X, U]
    if free_tf:
        parts.append(s.uniform(1, *d["tf"]))
    x = np.concatenate(parts)
    y = s.normal(m)
    vn = s.uniform(x.size, -1.0, 1.0)
    vm = s.normal(m)
    return dict(x=x, y=y, vn=vn, vm=vm)


def draw_batch_meta(seed: int, count: int, nmin: int, nmax: int):
    """Horizons N_i ~ U{nmin..nmax}, initial states ~ U(-0.5,0.5)^4, R_i ~ U(0.01,1)."""
    s = Stream(seed)
    Ns = s.integers(count, nmin, nmax)
    x0 = s.uniform(4 * count, -0.5, 0.5).reshape(count, 4)
    R = s.uniform(count, 0.01, 1.0)
    return Ns, x0, R


# Workload definitions (data only).  Model names: vdp, cartpole, heat, dint, quadrotor.
# Running cost f0 = sum_k q_k (x_k - xref_k(t))^2 + sum_i r_i (u_i - uref_i)^2, where the
# optional keys xslope, xamp, xfreq make the state reference time-varying:
# xref_k(t) = xref_k + xslope_k t + xamp_k sin(xfreq_k t).
def workload(name: str) -> dict:
    if name == "vdp_n1e3":         # Van der Pol, N=1000, T=10, x0=(1,0), cost x1^2+x2^2+u^2
        return dict(name=name, model="vdp", nx=2, nu=1, N=1000, T=10.0, params=[1.0],
                    q=[1.0, 1.0], r=[1.0], xref=[0.0, 0.0], uref=[0.0], x0=[1.0, 0.0], xf=None,
                    seed=1000, sigma=1.0, dist="vdp")
    if name == "cartpole_n1e5":    # cart-pole, mc=1, mp=0.1, l=0.5, g=9.81, N=1e5, T=5, Q=I4, R=0.1
        return dict(name=name, model="cartpole", nx=4, nu=1, N=100000, T=5.0,
                    params=[1.0, 0.1, 0.5, 9.81], q=[1.0] * 4, r=[0.1], xref=[0.0] * 4, uref=[0.0],
                    x0=[0.0] * 4, xf=None, seed=1001, sigma=1.0, dist="cartpole")
    if name == "heat_n2e4":        # heat, 64 cells, dx=1/64, N=2e4, T=1, cost ||x-0.5||^2 + 1e-2 u^2
        return dict(name=name, model="heat", nx=64, nu=1, N=20000, T=1.0, params=[64.0],
                    q=[1.0] * 64, r=[1e-2], xref=[0.5] * 64, uref=[0.0], x0=[0.0] * 64, xf=None,
                    seed=1002, sigma=1.0, dist="heat")
    if name == "vdp_mu_n1e6":      # Van der Pol with parameter mu, N=1e6, T=10
        return dict(name=name, model="vdp", nx=2, nu=1, N=1_000_000, T=10.0, params=[1.0],
                    q=[1.0, 1.0], r=[1.0], xref=[0.0, 0.0], uref=[0.0], x0=[1.0, 0.0], xf=None,
                    seed=1003, sigma=1.0, dist="vdp")
    if name == "cartpole_n1e6":    # the cart-pole at N=1e6
        w = workload("cartpole_n1e5")
        w.update(name=name, N=1_000_000, seed=1005)
        return w
    if name == "dint":             # double integrator, min 1/2 int u^2, x(0)=(-1,0), x(1)=(0,0)
        return dict(name=name, model="dint", nx=2, nu=1, N=100, T=1.0, params=[],
                    q=[0.0, 0.0], r=[0.5], xref=[0.0, 0.0], uref=[0.0], x0=[-1.0, 0.0],
                    xf=[0.0, 0.0], seed=1006, sigma=1.0, dist="dint")
    if name.startswith("quadrotor_n"):  # the paper's quadrotor (appendix): T=1, g=9.8, r=0.1
        N = {"quadrotor_n1e3": 1000, "quadrotor_n1e5": 100_000, "quadrotor_n1e6": 1_000_000}[name]
        T = 1.0
        # 1/2 [ (x1 - sin(2 pi t/T))^2 + (x3 - 2 sin(4 pi t/T))^2 + (x5 - 2 t/T)^2
        #       + x7^2 + x8^2 + x9^2 + r |u|^2 ]
        return dict(name=name, model="quadrotor", nx=9, nu=4, N=N, T=T, params=[9.8],
                    q=[0.5, 0.0, 0.5, 0.0, 0.5, 0.0, 0.5, 0.5, 0.5], r=[0.05] * 4,
                    xref=[0.0] * 9, uref=[0.0] * 4,
                    xslope=[0.0, 0.0, 0.0, 0.0, 2.0 / T, 0.0, 0.0, 0.0, 0.0],
                    xamp=[1.0, 0.0, 2.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0],
                    xfreq=[2.0 * np.pi / T, 0.0, 4.0 * np.pi / T, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0],
                    x0=[0.0] * 9, xf=None, seed={1000: 1007, 100_000: 1008, 1_000_000: 1009}[N],
                    sigma=1.0, dist="quadrotor")
    if name.startswith("goddard_n"):  # the paper's Goddard rocket (appendix), free final time
        N = {"goddard_n1e3": 1000, "goddard_n1e5": 100_000, "goddard_n1e6": 1_000_000}[name]
        inf = float("inf")
        # max r(tf)  s.t.  x(0) = (r0, v0, m0) = (1, 0, 1),  m(tf) = mf = 0.6,  0 <= u <= 1,
        # r >= r0,  0 <= v <= vmax = 0.1;  Cd = 310, beta = 500, Tmax = 3.5, b = 2; tf unbounded
        # (declared a real variable)
        return dict(name=name, model="goddard", nx=3, nu=1, N=N, T=1.0, params=[310.0, 500.0, 3.5, 2.0],
                    q=[0.0] * 3, r=[0.0], xref=[0.0] * 3, uref=[0.0], x0=[1.0, 0.0, 1.0],
                    xf=[0.6], xf_comp=[2], mayer=[-1.0, 0.0, 0.0], free_tf=True,
                    bounds=dict(xlo=[1.0, 0.0, -inf], xhi=[inf, 0.1, inf], ulo=[0.0], uhi=[1.0],
                                tflo=-inf, tfhi=inf),
                    seed={1000: 1010, 100_000: 1011, 1_000_000: 1012}[N], sigma=1.0, dist="goddard")
    raise KeyError(name)


# Path inequalities (paper Sec. 3: c(X_i, U_i) <= 0 at every node with a control), written as
# sum_v [a_v (z_v - b_v)^2 + l_v z_v] - r <= 0 over z = (x, u): one list entry per row.
def _path_rows(nz, rows):
    a = [[0.0] * nz for _ in rows]
    b = [[0.0] * nz for _ in rows]
    lin = [[0.0] * nz for _ in rows]
    r = []
    for i, (terms, rr) in enumerate(rows):
        for v, (av, bv, lv) in terms.items():
            a[i][v], b[i][v], lin[i][v] = av, bv, lv
        r.append(rr)
    return dict(a=a, b=b, l=lin, r=r)


PATHS = {
    # x2 >= -0.4 (the constrained Van der Pol problem) and u^2 <= 1
    "vdp": [({1: (0.0, 0.0, -1.0)}, 0.4), ({2: (1.0, 0.0, 0.0)}, 1.0)],
    # the cart within an ellipse in (p, theta), and F^2 <= 100
    "cartpole": [({0: (0.25, 0.0, 0.0), 2: (1.0, 0.0, 0.0)}, 1.0), ({4: (1.0, 0.0, 0.0)}, 100.0)],
    "dint": [({2: (1.0, 0.0, 0.0)}, 4.0)],
    # altitude band (x5 - 1)^2 <= 1, a keep-out disc around (x1, x3) = (0.5, 0.5) of radius 0.2,
    # and the tilt proxy x7^2 + x8^2 <= 0.5
    "quadrotor": [({4: (1.0, 1.0, 0.0)}, 1.0), ({0: (-1.0, 0.5, 0.0), 2: (-1.0, 0.5, 0.0)}, -0.04),
                  ({6: (1.0, 0.0, 0.0), 7: (1.0, 0.0, 0.0)}, 0.5)],
    # the speed limit v <= vmax as a constraint, and the thrust energy u^2 <= 1
    "goddard": [({1: (0.0, 0.0, 1.0)}, 0.1), ({3: (1.0, 0.0, 0.0)}, 1.0)],
    # the boundary control u^2 <= 1 and the first cell above 0 (x_1 >= 0)
    "heat": [({64: (1.0, 0.0, 0.0)}, 1.0), ({0: (0.0, 0.0, -1.0)}, 0.0)],
}


def with_path(w: dict) -> dict:
    """The workload with its model's path inequalities attached (key "path")."""
    return dict(w, path=_path_rows(w["nx"] + w["nu"], PATHS[w["model"]]))


# Boundary inequalities (paper Sec. 3: b(X_0, X_N) <= 0), in the same family as the path rows
# but over z = (X_0, X_N): index v < nx is X_{0,v}, nx + v is X_{N,v}.  One list per model,
# built for the workload's nx.
def _bineq_rows(model: str, nx: int):
    if model == "vdp":      # terminal ball |X_N|^2 <= 1/4, and X_{N,1} - X_{0,1} <= 1
        return [({2: (1.0, 0.0, 0.0), 3: (1.0, 0.0, 0.0)}, 0.25), ({0: (0.0, 0.0, -1.0), 2: (0.0, 0.0, 1.0)}, 1.0)]
    if model == "cartpole":  # the pole near upright at the end, the cart back within 0.5 of its start
        return [({nx + 2: (1.0, float(np.pi), 0.0)}, 0.01), ({0: (0.0, 0.0, -1.0), nx: (0.0, 0.0, 1.0)}, 0.5)]
    if model == "dint":     # final speed X_{N,2}^2 <= 0.01
        return [({nx + 1: (1.0, 0.0, 0.0)}, 0.01)]
    if model == "quadrotor":  # terminal position ball around (1, 1), altitude gain of at least 1
        return [({nx + 0: (1.0, 1.0, 0.0), nx + 2: (1.0, 1.0, 0.0)}, 0.1),
                ({4: (0.0, 0.0, 1.0), nx + 4: (0.0, 0.0, -1.0)}, -1.0)]
    if model == "goddard":  # altitude gain r(tf) - r(0) >= 1e-3, final speed v(tf)^2 <= 0.01
        return [({0: (0.0, 0.0, 1.0), nx + 0: (0.0, 0.0, -1.0)}, -1e-3), ({nx + 1: (1.0, 0.0, 0.0)}, 0.01)]
    if model == "heat":     # mean final temperature <= 0.6, last cell near 0.5 at the end
        return [({nx + k: (0.0, 0.0, 1.0 / nx) for k in range(nx)}, 0.6), ({2 * nx - 1: (1.0, 0.5, 0.0)}, 0.04)]
    raise KeyError(model)


def with_bineq(w: dict) -> dict:
    """The workload with its model's boundary inequalities attached (key "bineq")."""
    return dict(w, bineq=_path_rows(2 * w["nx"], _bineq_rows(w["model"], w["nx"])))


# Boundary cost (paper Sec. 3, the Bolza term g(X_0, X_N)) in the same family over
# z = (X_0, X_N): a terminal penalty 1.5 |X_N - b|^2 towards b_k = 0.1 (k + 1), a small quadratic
# and linear term on X_{0,1}, and a linear reward on X_{N,nx}.  With the Euler scheme (no
# Hessian block at node N) the X_N terms are linear only.
def with_bolza(w: dict) -> dict:
    nx = w["nx"]
    euler = w.get("scheme") == "euler"
    a = [0.0] * (2 * nx); b = [0.0] * (2 * nx); lin = [0.0] * (2 * nx)
    a[0], lin[0] = 0.5, -0.25
    for k in range(nx):
        if not euler:
            a[nx + k], b[nx + k] = 1.5, 0.1 * (k + 1)
    lin[2 * nx - 1] = 0.3
    return dict(w, bolza=dict(a=a, b=b, l=lin))


def with_horizon(w: dict, N: int) -> dict:
    """The same workload at another horizon (parity cases at oracle-friendly sizes)."""
    w = dict(w)
    w["N"] = int(N)
    return w


def final_rows(w: dict) -> int:
    """Number of final rows X_{N,k}: the listed components, or all when xf is given alone."""
    if w.get("xf_comp") is not None:
        return len(w["xf_comp"])
    return w["nx"] if w.get("xf") is not None else 0


def control_nodes(w: dict) -> int:
    """Nodes carrying a control: N + 1 (trapezoidal scheme) or N (forward Euler)."""
    return w["N"] if w.get("scheme") == "euler" else w["N"] + 1


def dims(w: dict):
    """(n, m) of the transcription: n = nx (N+1) + nu (controlled nodes) (+1 for a free final
    time); m = nx + final rows + nx N + path rows (one per inequality and controlled node)."""
    n = w["nx"] * (w["N"] + 1) + w["nu"] * control_nodes(w) + (1 if w.get("free_tf") else 0)
    npath = len(w["path"]["r"]) if w.get("path") else 0
    nbin = len(w["bineq"]["r"]) if w.get("bineq") else 0
    return n, w["nx"] + final_rows(w) + w["nx"] * w["N"] + npath * control_nodes(w) + nbin


def draw(w: dict, seed: int | None = None) -> dict:
    n, m = dims(w)
    return draw_instance(w["seed"] if seed is None else seed, w["dist"], w["nx"], w["nu"], w["N"], m,
                         free_tf=bool(w.get("free_tf")), unodes=control_nodes(w))


def batch_workloads(count=256, nmin=500, nmax=50000, seed=1004):
    """The batched cart-pole workload: `count` instances, N_i ~ U{nmin..nmax},
    x0_i ~ U(-0.5, 0.5)^4, R_i ~ U(0.01, 1); instance i draws its inputs with seed + 1 + i."""
    Ns, x0, R = draw_batch_meta(seed, count, nmin, nmax)
    base = workload("cartpole_n1e5")
    out = []
    for i in range(count):
        w = dict(base, name="cartpole_batch_%d" % i, N=int(Ns[i]), r=[float(R[i])], x0=[float(v) for v in x0[i]],
                 seed=seed + 1 + i)
        out.append(w)
    return out
