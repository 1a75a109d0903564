"""Seeded synthetic workloads shared by the CUDA path, the tests and the oracle.

This module holds workload descriptions (physical potentials, sizes, seeds) and
seeded input vectors only.  It holds none of the method's arithmetic: no index
set enumeration, no Chebyshev conversion, no coordinate matrices.  Functions that
need the multi-indices of an index set take them as an argument.

Axes are 0-based here (the paper counts them from 1).  A potential is the list of
components of W = V - 1/2 |x|^2 (Sec. 1.2, the harmonic part goes to D_K):

  {"coef": c, "powers": {axis: p, ...}, "mod": M}      c * prod x_axis^p * f(t)
  {"coef": c, "func": "cos_diff", "axes": [a, b], "R": R, "mod": M}
                                                        c * cos(x_a - x_b) * f(t)
  {"coef": c, "func": "cos_scaled", "axes": [a], "scale": s, "R": R, "mod": M}
                                                        c * cos(s * x_a) * f(t)

with the modulation f(t) given by M (default constant 1):
  {"kind": "const"} | {"kind": "cos", "omega": w, "phase": p}   (cos(w t + p))
  {"kind": "sin2", "omega": w}                                    (sin^2(w t))
  {"kind": "pwconst", "values": [...], "t0": a, "t1": b}          (piecewise constant)
"""
from __future__ import annotations

import math

import numpy as np


def half_width(B: int) -> float:
    """Domain half-width L = sqrt(2B) + 1, so that SL >= sqrt(2(K+1)) + 1 holds with S = 1 (Sec. 1.4)."""
    return math.sqrt(2.0 * B) + 1.0


def henon_heiles_chain(N: int, lam: float, dipole: tuple | None = None) -> list:
    """W = lam * sum_{d} (x_d^2 x_{d+1} - x_{d+1}^3 / 3) [+ E0 cos(w t) x_1]."""
    comps = []
    for d in range(N - 1):
        comps.append({"coef": lam, "powers": {d: 2, d + 1: 1}})
        comps.append({"coef": -lam / 3.0, "powers": {d + 1: 3}})
    if dipole is not None:
        e0, omega = dipole
        comps.append({"coef": e0, "powers": {0: 1}, "mod": {"kind": "cos", "omega": omega, "phase": 0.0}})
    return comps


def stretched_hh_laser(N: int, L: float) -> list:
    """sum_l [(x_l/L)^2 (x_{l+1}/L) - (x_{l+1}/L)^3 / 3] - sin^2(t) (x_1/L): the time-integration
    experiment's potential (Sec. 6.3), read with the laser term scaled like the others and without a
    -(1/2)|x|^2 term (the harmonic part stays in D_K)."""
    comps = []
    for d in range(N - 1):
        comps.append({"coef": 1.0 / L ** 3, "powers": {d: 2, d + 1: 1}})
        comps.append({"coef": -1.0 / (3.0 * L ** 3), "powers": {d + 1: 3}})
    comps.append({"coef": -1.0 / L, "powers": {0: 1}, "mod": {"kind": "sin2", "omega": 1.0}})
    return comps


def time_integration_workload(N: int, K: int, m: int = 7) -> dict:
    """The time-integration experiment of Sec. 6.3: K + 1 = B, L = 16, initial coefficients
    prod_{k_l != 0} k_l^-3 normalised, propagated over [0, 1]."""
    return dict(name=f"hhlaser{N}_k{K}", N=N, B=K + 1, L=16.0, potential=stretched_hh_laser(N, 16.0),
                desc="stretched Henon-Heiles, L = 16, - sin^2(t) x1 / L",
                init={"kind": "beta_decay", "beta": 3.0}, T=1.0, m=m)


def drifting_cos_chain(N: int, beta: float, omega: float, R: int = 8) -> list:
    """W(x, t) = beta * sum_d cos(x_d - x_{d+1} + omega t) + beta / 2 * cos(x_1 / 4 + omega t): a
    potential whose shape, not only its size, changes with t, so that its degree-R Chebyshev
    interpolant has to be computed anew for every time step."""
    comps = [{"coef": beta, "func": "cos_diff", "axes": [d, d + 1], "R": R, "omega": omega} for d in range(N - 1)]
    comps.append({"coef": 0.5 * beta, "func": "cos_scaled", "axes": [0], "scale": 0.25, "R": R, "omega": omega})
    return comps


def cos_chain(N: int, beta: float, R: int = 8) -> list:
    """W = beta * sum_d cos(x_d - x_{d+1}), to be replaced by its degree-R Chebyshev interpolant."""
    return [{"coef": beta, "func": "cos_diff", "axes": [d, d + 1], "R": R} for d in range(N - 1)]


def control_quartic(u_values, t_end: float) -> list:
    """W = 0.1 x_1^2 x_2^2 + u(t) x_1 with u piecewise constant on len(u_values) intervals of [0, t_end]."""
    return [
        {"coef": 0.1, "powers": {0: 2, 1: 2}},
        {"coef": 1.0, "powers": {0: 1},
         "mod": {"kind": "pwconst", "values": [float(u) for u in u_values], "t0": 0.0, "t1": float(t_end)}},
    ]


def workload(name: str) -> dict:
    """The named synthetic workloads (sizes, potentials, seeds, step parameters)."""
    if name == "hh2_b32":          # N=2 Henon-Heiles, FP64, 100 steps
        N, B = 2, 32
        return dict(name=name, N=N, B=B, L=half_width(B), potential=henon_heiles_chain(N, 0.111),
                    desc="Henon-Heiles lambda=0.111",
                    init={"kind": "coherent", "q": [1.0, 1.0], "eps": 1e-3, "seed": 0},
                    dt=0.01, steps=100, m=7)
    if name == "hh6_b4096":        # N=6 Henon-Heiles chain + dipole, 1000 steps
        N, B = 6, 4096
        return dict(name=name, N=N, B=B, L=half_width(B),
                    potential=henon_heiles_chain(N, 0.111, dipole=(0.05, 1.0)),
                    desc="Henon-Heiles chain lambda=0.111 + 0.05 cos(t) x1",
                    init={"kind": "gaussian", "seed": 1}, dt=0.01, steps=1000, m=7,
                    dt_converged=2.5e-5)   # each m = 7 exponential within the estimate 1e-6 (about 4e-8)
    if name == "cos10_b1024":      # N=10 cosine chain, degree-8 interpolant, 500 steps
        N, B = 10, 1024
        return dict(name=name, N=N, B=B, L=half_width(B), potential=cos_chain(N, 0.2, 8),
                    desc="0.2 sum cos(x_d - x_{d+1}), degree-8 Chebyshev interpolant",
                    init={"kind": "decaying", "seed": 2, "power": 2.0}, dt=0.01, steps=500, m=7,
                    dt_converged=1e-3)   # ||A|| about 5e2 (the diagonal): h ||A|| about 0.5
    if name == "ctrl4_b512":       # N=4 control problem for the adjoint gradient
        N, B = 4, 512
        rng = np.random.default_rng(4)
        u = rng.uniform(-0.1, 0.1, size=200)
        return dict(name=name, N=N, B=B, L=half_width(B), potential=control_quartic(u, 10.0),
                    desc="0.1 x1^2 x2^2 + u(t) x1, u piecewise constant on 200 intervals",
                    init={"kind": "coherent", "q": [1.0, 0.0, 0.0, 0.0], "eps": 0.0, "seed": 4},
                    T=10.0, intervals=200, substeps=10, target=[1, 0, 0, 0], u=u.tolist(), m=7)
    if name == "hh6_b32768":       # roofline size: one vector well above L2
        N, B = 6, 32768
        return dict(name=name, N=N, B=B, L=half_width(B),
                    potential=henon_heiles_chain(N, 0.111, dipole=(0.05, 1.0)),
                    desc="Henon-Heiles chain lambda=0.111 + 0.05 cos(t) x1",
                    init={"kind": "gaussian", "seed": 1}, dt=0.01, steps=10, m=7)
    raise KeyError(name)


def batch_workloads(n: int = 256, seed: int = 3, b_lo: int = 64, b_hi: int = 8192) -> list:
    """Independent Henon-Heiles problems: N ~ U{2..8}, B log-uniform in [b_lo, b_hi],
    lambda ~ U[0.05, 0.15], coherent-state centres q ~ U[-1, 1]^N."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        N = int(rng.integers(2, 9))
        B = int(round(math.exp(rng.uniform(math.log(b_lo), math.log(b_hi)))))
        lam = float(rng.uniform(0.05, 0.15))
        q = rng.uniform(-1.0, 1.0, size=N).tolist()
        out.append(dict(name=f"batch{i}", N=N, B=B, L=half_width(B), potential=henon_heiles_chain(N, lam),
                        init={"kind": "coherent", "q": q, "eps": 0.0, "seed": 1000 + i}, dt=0.01, m=7))
    return out


# --------------------------------------------------------------------------- #
# seeded vectors                                                               #
# --------------------------------------------------------------------------- #

def complex_gaussian(n: int, seed: int) -> np.ndarray:
    """iid complex Gaussian entries, real and imaginary parts each N(0, 1), unnormalised."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


def coherent_state(kidx: np.ndarray, q) -> np.ndarray:
    """Hermite coefficients of the unit-width Gaussian pi^{-N/4} exp(-|x - q|^2 / 2) (momentum 0):
    c_k = prod_l exp(-q_l^2 / 4) (q_l / sqrt 2)^{k_l} / sqrt(k_l!)."""
    kidx = np.asarray(kidx, dtype=np.int64)
    out = np.ones(kidx.shape[0])
    for l, ql in enumerate(q):
        kl = kidx[:, l]
        kmax = int(kl.max()) if kl.size else 0
        tab = np.empty(kmax + 1)
        tab[0] = math.exp(-ql * ql / 4.0)
        for k in range(1, kmax + 1):
            tab[k] = tab[k - 1] * (ql / math.sqrt(2.0)) / math.sqrt(k)
        out *= tab[kl]
    return out.astype(np.complex128)


def lex_sorted(ks: np.ndarray) -> np.ndarray:
    """Rows of ks in lexicographic order, last coordinate fastest (the canonical order)."""
    ks = np.asarray(ks, dtype=np.int32)
    return ks[np.lexsort(ks.T[::-1])]


def total_degree_set(N: int, K: int) -> np.ndarray:
    """The total-degree set {k in N^N : k_1 + ... + k_N <= K}, a downward-closed set (Sec. 1.2)."""
    out = []

    def rec(prefix, left):
        if len(prefix) == N:
            out.append(list(prefix))
            return
        for k in range(left + 1):
            rec(prefix + [k], left - k)

    rec([], K)
    return lex_sorted(np.array(out, dtype=np.int32))


def random_downward_closed_set(N: int, size: int, seed: int) -> np.ndarray:
    """A seeded random downward-closed set of the given size: starting from {0}, repeatedly add a
    uniformly chosen point outside the set all of whose lower neighbours k - e_l are in it."""
    rng = np.random.default_rng(seed)
    members = {(0,) * N}
    frontier = {tuple(1 if l == i else 0 for l in range(N)) for i in range(N)}
    while len(members) < size:
        cand = sorted(frontier)
        k = cand[int(rng.integers(len(cand)))]
        frontier.discard(k)
        members.add(k)
        for l in range(N):
            up = tuple(k[i] + (1 if i == l else 0) for i in range(N))
            if up not in members and all(tuple(up[i] - (1 if i == d else 0) for i in range(N)) in members
                                         for d in range(N) if up[d] > 0):
                frontier.add(up)
    return lex_sorted(np.array(sorted(members), dtype=np.int32))


def initial_vector(spec: dict, kidx: np.ndarray) -> np.ndarray:
    """The normalised initial coefficient vector of a workload, in canonical order of kidx."""
    init = spec["init"]
    n = kidx.shape[0]
    if init["kind"] == "gaussian":
        c = complex_gaussian(n, init["seed"])
    elif init["kind"] == "coherent":
        c = coherent_state(kidx, init["q"])
        if init.get("eps", 0.0):
            c = c / np.linalg.norm(c) + init["eps"] * complex_gaussian(n, init["seed"])
    elif init["kind"] == "decaying":
        w = np.prod(1.0 + np.asarray(kidx, dtype=np.float64), axis=1) ** (-init["power"])
        c = complex_gaussian(n, init["seed"]) * w
    elif init["kind"] == "beta_decay":   # v_k = prod max(k_l, 1)^-beta (Sec. 6.1)
        c = np.prod(np.maximum(np.asarray(kidx, dtype=np.float64), 1.0), axis=1) ** (-init["beta"])
        c = c.astype(np.complex128)
    else:
        raise KeyError(init["kind"])
    return c / np.linalg.norm(c)


def sample_rows(n: int, count: int, seed: int = 7) -> np.ndarray:
    """Sorted distinct row indices for sampled parity checks, always including 0 and n-1."""
    rng = np.random.default_rng(seed)
    count = min(count, n)
    rows = set(rng.choice(n, size=count, replace=False).tolist())
    rows.update({0, n - 1})
    return np.array(sorted(rows), dtype=np.int64)
