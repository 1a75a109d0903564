"""ORACLE — test infrastructure only.

Plain, slow FP64 CPU restatement of Brumm, "A fast matrix-free algorithm for
spectral approximations to the Schroedinger equation" (arXiv:1403.3511).  It is
independent of the CUDA library: it neither imports it nor shares any code,
table or constant generator with it.  Only tests/, __graft_entry__.smoke() and
the cpu_baseline / reference legs of bench.py may import it.

Layout
  - hx_oracle.c (loaded through ctypes): index sets, direct_op, the Chebyshev
    recurrence and the fast algorithm, literally and term by term (Sec. 3).
  - this file: Chebyshev interpolation of W (Sec. 1.3), dense coordinate
    matrices for tiny sets, Gauss-Hermite assembly (Sec. 4), Hermitian Lanczos
    for the exponential (Sec. 2.2), the exponential midpoint rule (Sec. 2.1),
    and the FP64 adjoint gradient for a piecewise-constant control.

Readings of the paper that the oracle fixes (each also listed in the design notes):
  - index set: {k : prod(1 + k_l) <= B}, B = K + 1 (Sec. 1.2);
  - direct_op drops v_{j+e_l} exactly when j + e_l is not in the set;
  - factor order inside a product: "sym", the mean of the order of Eq. (Horner)
    and the order of Algorithm fast_algorithm (both kept as "eq" / "alg");
  - each term of the fast algorithm restarts from the input vector;
  - Chebyshev nodes of the first kind, R + 1 nodes for degree R;
  - Lanczos: full reorthogonalisation by classical Gram-Schmidt applied twice;
  - time-dependent potentials are interpolated anew at every time an integrator
    evaluates A (the time-propagation algorithm of Sec. 2.2, step (1)).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from typing import Callable

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_hx_oracle.so")
_ORDERS = {"sym": 0, "eq": 1, "alg": 2}


def build() -> str:
    """Compile hx_oracle.c with gcc (plain C99, -O2, no target-specific flags)."""
    src = os.path.join(_HERE, "hx_oracle.c")
    if (not os.path.exists(_SO)) or os.path.getmtime(_SO) < max(os.path.getmtime(src),
                                                                 os.path.getmtime(os.path.join(_HERE, "hx_oracle.h"))):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", src, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        L.ho_hc_count.restype = i64
        L.ho_hc_count.argtypes = [ctypes.c_int, i64]
        L.ho_hc_create.restype = P
        L.ho_hc_create.argtypes = [ctypes.c_int, i64]
        L.ho_list_create.restype = P
        L.ho_list_create.argtypes = [ctypes.c_int, i64, P]
        L.ho_set_free.argtypes = [P]
        L.ho_set_k.restype = P
        L.ho_set_k.argtypes = [P]
        L.ho_set_size.restype = i64
        L.ho_set_size.argtypes = [P]
        L.ho_rank.restype = i64
        L.ho_rank.argtypes = [P, P]
        L.ho_neighbors_build.argtypes = [P]
        L.ho_direct_op.argtypes = [P, ctypes.c_int, P, P]
        L.ho_cheb_apply.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_double, P, P]
        L.ho_fast_algorithm.argtypes = [P, ctypes.c_int, P, P, ctypes.c_double, ctypes.c_int, P, P]
        L.ho_diag_apply.argtypes = [P, P, P]
        L.ho_apply.argtypes = [P, ctypes.c_int, P, P, ctypes.c_double, ctypes.c_int, P, P]
        L.ho_apply_rows_local.argtypes = [P, i64, ctypes.c_int, P, P, ctypes.c_double, ctypes.c_int, P, i64, P, P]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class IndexSet:
    """A finite multi-index set in lexicographic order, last coordinate fastest (Sec. 1.2)."""

    def __init__(self, handle, N: int, B: int | None):
        self._h = handle
        self.N = N
        self.B = B
        self.size = int(lib().ho_set_size(handle))
        buf = lib().ho_set_k(handle)
        n = self.size * N
        self.k = np.ctypeslib.as_array((ctypes.c_int32 * max(n, 1)).from_address(buf))[:n].reshape(self.size, N)

    @classmethod
    def hyperbolic(cls, N: int, B: int) -> "IndexSet":
        """{k in N^N : prod_l (1 + k_l) <= B}, the hyperbolically reduced set with K + 1 = B (Sec. 1.2)."""
        h = lib().ho_hc_create(N, B)
        if not h:
            raise ValueError("bad N or B")
        return cls(h, N, B)

    @classmethod
    def full(cls, N: int, K: int) -> "IndexSet":
        """K_full(K) = {k : 0 <= k_l <= K} (Sec. 1.2)."""
        grids = np.meshgrid(*[np.arange(K + 1)] * N, indexing="ij")
        ks = np.stack([g.ravel() for g in grids], axis=1).astype(np.int32)
        return cls.from_list(ks)

    @classmethod
    def from_list(cls, ks: np.ndarray) -> "IndexSet":
        ks = np.ascontiguousarray(ks, dtype=np.int32)
        h = lib().ho_list_create(ks.shape[1], ks.shape[0], _ptr(ks))
        if not h:
            raise ValueError("index list must be strictly increasing in lexicographic order")
        return cls(h, ks.shape[1], None)

    def rank(self, k) -> int:
        kk = np.ascontiguousarray(k, dtype=np.int32)
        return int(lib().ho_rank(self._h, _ptr(kk)))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.ho_set_free(self._h)
            self._h = None


def hc_count(N: int, B: int) -> int:
    return int(lib().ho_hc_count(N, B))


# --------------------------------------------------------------------------- #
# Chebyshev interpolation of W (Sec. 1.3)                                      #
# --------------------------------------------------------------------------- #

def cheb_nodes(R: int) -> np.ndarray:
    """First-kind Chebyshev nodes u_i = cos(pi (2i + 1) / (2R + 2)), i = 0..R, on [-1, 1]."""
    i = np.arange(R + 1)
    return np.cos(np.pi * (2 * i + 1) / (2 * R + 2))


def cheb_coeffs_1d(values: np.ndarray) -> np.ndarray:
    """Coefficients a_r of the interpolant sum_r a_r T_r through values at cheb_nodes(R):
    a_r = (2 - delta_{r0}) / (R + 1) * sum_i f(u_i) cos(r theta_i)  (discrete orthogonality of T_r)."""
    R = len(values) - 1
    theta = np.pi * (2 * np.arange(R + 1) + 1) / (2 * R + 2)
    a = np.array([np.sum(values * np.cos(r * theta)) for r in range(R + 1)]) * (2.0 / (R + 1))
    a[0] /= 2.0
    return a


def cheb_coeffs_2d(values: np.ndarray) -> np.ndarray:
    """Tensor-product version of cheb_coeffs_1d: values[i, j] = f(u_i, u_j)."""
    R = values.shape[0] - 1
    theta = np.pi * (2 * np.arange(R + 1) + 1) / (2 * R + 2)
    C = np.cos(np.outer(np.arange(R + 1), theta)) * (2.0 / (R + 1))
    C[0] /= 2.0
    return C @ values @ C.T


def potential_terms(spec: dict, t: float) -> tuple[np.ndarray, np.ndarray]:
    """alpha_r(t) of W^pol(x, t) = sum_r alpha_r(t) T_r(x / L) for a workload's potential (Sec. 1.3).

    Every component is interpolated on [-L, L]^axes at Chebyshev nodes of the first kind, at the
    time t (a component whose function itself depends on t, "omega" != 0, is interpolated anew
    for every t); a monomial is interpolated at its own degree per axis, which reproduces it
    exactly.
    Returns (r, alpha) with r of shape (nterms, N), duplicates merged, zeros dropped."""
    N, L = spec["N"], spec["L"]
    acc: dict[tuple, float] = {}
    for comp in spec["potential"]:
        f_t = modulation(comp.get("mod", {"kind": "const"}), t) * comp["coef"]
        if f_t == 0.0:
            continue
        if "powers" in comp:
            axes = sorted(comp["powers"])
            degs = [comp["powers"][a] for a in axes]
            per_axis = []
            for p in degs:   # x^p = L^p u^p, interpolated at degree p (exact)
                u = cheb_nodes(p)
                per_axis.append(cheb_coeffs_1d((L * u) ** p))
            for idx in np.ndindex(*[p + 1 for p in degs]):
                a = f_t * np.prod([per_axis[i][idx[i]] for i in range(len(axes))])
                r = [0] * N
                for i, ax in enumerate(axes):
                    r[ax] = idx[i]
                acc[tuple(r)] = acc.get(tuple(r), 0.0) + a
        elif comp["func"] == "cos_diff":
            a_ax, b_ax = comp["axes"]
            R = comp["R"]
            u = cheb_nodes(R)
            vals = np.cos(L * u[:, None] - L * u[None, :] + comp.get("omega", 0.0) * t)
            coef = cheb_coeffs_2d(vals) * f_t
            for i in range(R + 1):
                for j in range(R + 1):
                    r = [0] * N
                    r[a_ax], r[b_ax] = i, j
                    acc[tuple(r)] = acc.get(tuple(r), 0.0) + coef[i, j]
        elif comp["func"] == "cos_scaled":
            (ax,) = comp["axes"]
            R = comp["R"]
            u = cheb_nodes(R)
            coef = cheb_coeffs_1d(np.cos(comp["scale"] * L * u + comp.get("omega", 0.0) * t)) * f_t
            for i in range(R + 1):
                r = [0] * N
                r[ax] = i
                acc[tuple(r)] = acc.get(tuple(r), 0.0) + coef[i]
        else:
            raise KeyError(comp["func"])
    keys = [k for k, v in acc.items() if v != 0.0]
    keys.sort()
    r = np.array(keys, dtype=np.int32).reshape(len(keys), N)
    alpha = np.array([acc[k] for k in keys], dtype=np.float64)
    return r, alpha


def modulation(mod: dict, t: float) -> float:
    kind = mod["kind"]
    if kind == "const":
        return 1.0
    if kind == "cos":
        return math.cos(mod["omega"] * t + mod.get("phase", 0.0))
    if kind == "sin2":
        return math.sin(mod["omega"] * t) ** 2
    if kind == "pwconst":
        vals = mod["values"]
        n = len(vals)
        q = int(math.floor((t - mod["t0"]) / (mod["t1"] - mod["t0"]) * n))
        return float(vals[min(max(q, 0), n - 1)])
    raise KeyError(kind)


# --------------------------------------------------------------------------- #
# the operator (Sec. 3)                                                        #
# --------------------------------------------------------------------------- #

def direct_op(S: IndexSet, l: int, v: np.ndarray) -> np.ndarray:
    v = np.ascontiguousarray(v, dtype=np.complex128)
    out = np.empty_like(v)
    lib().ho_direct_op(S._h, l, _ptr(v), _ptr(out))
    return out


def fast_algorithm(S: IndexSet, r: np.ndarray, alpha: np.ndarray, L: float, v: np.ndarray,
                   order: str = "sym") -> np.ndarray:
    """W^pol(X_K) v, Eq. (Horner), term by term (Algorithm fast_algorithm)."""
    v = np.ascontiguousarray(v, dtype=np.complex128)
    r = np.ascontiguousarray(r, dtype=np.int32)
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    out = np.empty_like(v)
    if lib().ho_fast_algorithm(S._h, len(alpha), _ptr(r), _ptr(alpha), L, _ORDERS[order], _ptr(v), _ptr(out)):
        raise MemoryError
    return out


def apply(S: IndexSet, r: np.ndarray, alpha: np.ndarray, L: float, v: np.ndarray, order: str = "sym",
          scale: float = 1.0) -> np.ndarray:
    """A(t) v = D_K v + W^pol(X_K, t) v, the right-hand side of Eq. (ODECoefficientsPol).

    scale = S != 1: the basis of scaled Hermite functions phi_k(S x) (Sec. 1.4).  With y = S x the
    Hamiltonian is S^2 (-1/2 Laplacian_y) + V(y / S), -1/2 Laplacian_y = H_osc - |y|^2 / 2 with H_osc
    diagonal (D_K) in this basis, and V = |x|^2 / 2 + W, so
      A = S^2 D_K + (1/S^2 - S^2)/2 sum_l X_l X_l + W(X / S),
    X_l the truncated coordinate matrices; W's Chebyshev terms in x / L are terms in y / (S L)."""
    v = np.ascontiguousarray(v, dtype=np.complex128)
    if scale != 1.0:
        out = scale ** 2 * diag(S) * v + fast_algorithm(S, r, alpha, L * scale, v, order)
        c = 0.5 * (1.0 / scale ** 2 - scale ** 2)
        for l in range(S.N):
            out += c * direct_op(S, l, direct_op(S, l, v))
        return out
    r = np.ascontiguousarray(r, dtype=np.int32)
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    out = np.empty_like(v)
    if lib().ho_apply(S._h, len(alpha), _ptr(r), _ptr(alpha), L, _ORDERS[order], _ptr(v), _ptr(out)):
        raise MemoryError
    return out


def apply_rows(S: IndexSet, B: int, r: np.ndarray, alpha: np.ndarray, L: float, c: np.ndarray,
               rows: np.ndarray, order: str = "sym") -> np.ndarray:
    """Entries (A(t) c)_j for the given rows only, each from a local window (hx_oracle.c)."""
    c = np.ascontiguousarray(c, dtype=np.complex128)
    r = np.ascontiguousarray(r, dtype=np.int32)
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.empty(len(rows), dtype=np.complex128)
    if lib().ho_apply_rows_local(S._h, B, len(alpha), _ptr(r), _ptr(alpha), L, _ORDERS[order],
                                 _ptr(c), len(rows), _ptr(rows), _ptr(out)):
        raise IndexError("row out of range")
    return out


def diag(S: IndexSet) -> np.ndarray:
    """Diagonal of D_K: sum_l (k_l + 1/2) (Sec. 1.2)."""
    return S.k.astype(np.float64).sum(axis=1) + 0.5 * S.N


# --------------------------------------------------------------------------- #
# dense matrices for tiny sets                                                 #
# --------------------------------------------------------------------------- #

def dense_X(S: IndexSet, l: int) -> np.ndarray:
    """(X_K^{(l)})_{jk} = (phi_j, x_l phi_k) from the recurrence Eq. (Recurrence1D):
    sqrt((k_l+1)/2) where j = k + e_l and sqrt(k_l/2) where j = k - e_l, both in the set."""
    n = S.size
    X = np.zeros((n, n))
    lookup = {tuple(k): i for i, k in enumerate(S.k.tolist())}
    for i, k in enumerate(S.k.tolist()):
        kp = list(k)
        kp[l] += 1
        jp = lookup.get(tuple(kp))
        if jp is not None:
            X[jp, i] = math.sqrt((k[l] + 1) / 2.0)
            X[i, jp] = math.sqrt((k[l] + 1) / 2.0)
    return X


def dense_cheb(X: np.ndarray, r: int, L: float) -> np.ndarray:
    """T_r(X / L) as a dense matrix by the recurrence Eq. (ChebyshevRecurrence)."""
    n = X.shape[0]
    t0, t1 = np.eye(n), X / L
    if r == 0:
        return t0
    for _ in range(r - 1):
        t0, t1 = t1, 2.0 * (X / L) @ t1 - t0
    return t1


def dense_W(S: IndexSet, r: np.ndarray, alpha: np.ndarray, L: float, order: str = "sym") -> np.ndarray:
    """Dense W^pol(X_K) of Eq. (Horner) with the factor order of the fast algorithm."""
    N, n = S.N, S.size
    Xs = [dense_X(S, l) for l in range(N)]
    W = np.zeros((n, n))
    for rt, a in zip(np.asarray(r).tolist(), np.asarray(alpha).tolist()):
        F = [dense_cheb(Xs[l], rt[l], L) for l in range(N)]
        eq = np.eye(n)      # T_{r_1}(X1) ... T_{r_N}(XN): axis N acts on v first
        for l in range(N):
            eq = eq @ F[l]
        alg = np.eye(n)     # axis 1 acts on v first
        for l in range(N):
            alg = F[l] @ alg
        W += a * {"eq": eq, "alg": alg, "sym": 0.5 * (eq + alg)}[order]
    return W


def dense_A(S: IndexSet, r, alpha, L, order="sym", scale: float = 1.0) -> np.ndarray:
    """The matrix of apply (dense), in the basis phi_k(scale x)."""
    if scale == 1.0:
        return np.diag(diag(S)) + dense_W(S, r, alpha, L, order)
    c = 0.5 * (1.0 / scale ** 2 - scale ** 2)
    A = np.diag(scale ** 2 * diag(S)) + dense_W(S, r, alpha, L * scale, order)
    for l in range(S.N):
        X = dense_X(S, l)
        A += c * (X @ X)
    return A


# --------------------------------------------------------------------------- #
# Gauss-Hermite assembly (Sec. 4)                                              #
# --------------------------------------------------------------------------- #

def hermite_functions_scaled(kmax: int, x: np.ndarray) -> np.ndarray:
    """h_k(x) = phi_k(x) exp(x^2 / 2) for k = 0..kmax by Eq. (Recurrence1D), starting from
    phi_0 = pi^{-1/4} exp(-x^2/2); returns an array of shape (kmax + 1, len(x))."""
    h = np.zeros((kmax + 1, len(x)))
    h[0] = math.pi ** -0.25
    if kmax >= 1:
        h[1] = x * h[0] / math.sqrt(0.5)
    for k in range(1, kmax):
        h[k + 1] = (x * h[k] - math.sqrt(k / 2.0) * h[k - 1]) / math.sqrt((k + 1) / 2.0)
    return h


def gh_factor_tables(kmax: int, rmax: int, L: float, M: int):
    """Per-axis tables G[r][j, k] = sum_m omega_m phi_j(xi_m) T_r(xi_m / L) phi_k(xi_m) with the
    (M+1)-point Gauss-Hermite rule (xi_m zeros of H_{M+1}, omega_m = w_m exp(xi_m^2)), Eq. (GHQuad_full)."""
    xi, w = np.polynomial.hermite.hermgauss(M + 1)
    h = hermite_functions_scaled(kmax, xi)
    T = np.zeros((rmax + 1, len(xi)))
    T[0] = 1.0
    if rmax >= 1:
        T[1] = xi / L
    for r in range(1, rmax):
        T[r + 1] = 2.0 * (xi / L) * T[r] - T[r - 1]
    return np.einsum("m,jm,rm,km->rjk", w, h, T, h)


def gh_assembly(S: IndexSet, r: np.ndarray, alpha: np.ndarray, L: float, M: int) -> np.ndarray:
    """W^{GH(M)}_{K,pol} with entries sum_r alpha_r prod_l G_l[r_l][j_l, k_l], Eq. (GHQuad_full)."""
    N = S.N
    kmax = int(S.k.max())
    rmax = int(np.max(r)) if len(r) else 0
    G = gh_factor_tables(kmax, rmax, L, M)
    n = S.size
    W = np.zeros((n, n))
    K = S.k
    for rt, a in zip(np.asarray(r).tolist(), np.asarray(alpha).tolist()):
        P = np.full((n, n), a)
        for l in range(N):
            P = P * G[rt[l]][np.ix_(K[:, l], K[:, l])]
        W += P
    return W


# --------------------------------------------------------------------------- #
# time integration (Sec. 2)                                                    #
# --------------------------------------------------------------------------- #

def lanczos_exp(apply_fn: Callable[[np.ndarray], np.ndarray], c: np.ndarray, h: float, m: int,
                breakdown: float = 1e-13, estimate: bool = False):
    """exp(-i h A) c ~ beta_0 V_m exp(-i h T_m) e_1 with an m-step Hermitian Lanczos process
    (Sec. 2.2), started from v_1 = c / ||c||.  Each new vector is orthogonalised against all
    previous ones by classical Gram-Schmidt, applied twice; T_m's diagonal holds the summed
    projections on v_k, its off-diagonal the norms.  Stops early when beta_k falls below
    breakdown * max_i(|alpha_i| + beta_i).  Returns (c_new, alphas, betas).

    estimate=True also returns the a-posteriori estimate of the relative error: the Lanczos
    relation A V_m = V_m T_m + beta_m v_{m+1} e_m^T leaves the residual beta_m v_{m+1} e_m^T, and
    the estimate is |h| beta_m |e_m^T exp(-i h T_m) e_1| with beta_m the norm of the m-th vector's
    remainder after its two orthogonalisations (0 after an early stop: the space is invariant)."""
    beta0 = np.linalg.norm(c)
    n = c.shape[0]
    V = np.zeros((m, n), dtype=np.complex128)
    V[0] = c / beta0
    alphas, betas = [], []
    scale = 0.0
    for k in range(m):
        w = apply_fn(V[k])
        a_k = 0.0
        for _ in range(2):
            coeffs = V[: k + 1].conj() @ w
            w = w - coeffs @ V[: k + 1]
            a_k += coeffs[k].real
        alphas.append(a_k)
        scale = max(scale, abs(a_k) + (betas[-1] if betas else 0.0))
        b_k = float(np.linalg.norm(w))
        if k == m - 1:
            beta_m = b_k if b_k > breakdown * scale else 0.0
            break
        if b_k <= breakdown * scale:
            beta_m = 0.0
            break
        betas.append(b_k)
        V[k + 1] = w / b_k
    mm = len(alphas)
    T = np.diag(alphas) + np.diag(betas[: mm - 1], 1) + np.diag(betas[: mm - 1], -1)
    lam, Q = np.linalg.eigh(T)
    y = Q @ (np.exp(-1j * h * lam) * Q[0, :])
    out = (beta0 * (y @ V[:mm]), np.array(alphas), np.array(betas[: mm - 1]))
    if estimate:
        return out + (abs(h) * beta_m * abs(y[mm - 1]) if mm == m else 0.0,)
    return out


def expmpr_propagate(S: IndexSet, spec: dict, c0: np.ndarray, h: float, nsteps: int, m: int,
                     t0: float = 0.0, order: str = "sym"):
    """c^{n+1} = exp(-i h A(t^n + h/2)) c^n, Eq. (expMPR), each exponential by lanczos_exp."""
    c = np.array(c0, dtype=np.complex128)
    t = t0
    for _ in range(nsteps):
        r, alpha = potential_terms(spec, t + 0.5 * h)
        c, _, _ = lanczos_exp(lambda v: apply(S, r, alpha, spec["L"], v, order, spec.get("scale", 1.0)), c, h, m)
        t += h
    return c, t


def galerkin_reference(S: IndexSet, spec: dict, c0: np.ndarray, T: float, M: int | None = None) -> np.ndarray:
    """c(T) for i c' = (D_K + W_K(t)) c with the exact Galerkin matrix W_K(t) of W^pol(., t) on K
    (not the fast algorithm's W^pol(X_K, t)): Gauss-Hermite assembly, Eq. (GHQuad_full), with M + 1
    >= K + R/2 + 2 nodes, which integrates every entry exactly for these polynomial degrees; the ODE is
    integrated by scipy's DOP853 at rtol 1e-13.  The potential's time dependence must be a modulation
    of whole components (W(t) = W_0 + sum_j f_j(t) W_j).  Tiny sets only (dense matrices)."""
    from scipy.integrate import solve_ivp
    kmax = int(S.k.max())
    M = M if M is not None else kmax + 6
    groups = {}
    for comp in spec["potential"]:
        key = repr(comp.get("mod", {"kind": "const"}))
        groups.setdefault(key, []).append(comp)
    mats = []
    for key, comps in groups.items():
        mod = comps[0].get("mod", {"kind": "const"})
        sub = dict(spec, potential=[dict(c, mod={"kind": "const"}) for c in comps])
        r, a = potential_terms(sub, 0.0)
        mats.append((mod, gh_assembly(S, r, a, spec["L"], M) if len(r) else np.zeros((S.size, S.size))))
    D = np.diag(diag(S))

    def rhs(t, y):
        A = D.copy()
        for mod, W in mats:
            A += modulation(mod, t) * W
        return -1j * (A @ y)

    sol = solve_ivp(rhs, (0.0, T), np.asarray(c0, dtype=np.complex128), method="DOP853", rtol=1e-13, atol=1e-15)
    return sol.y[:, -1]


MAGNUS4_NODES = (0.5 - np.sqrt(3.0) / 6.0, 0.5 + np.sqrt(3.0) / 6.0)


def magnus4_propagate(S: IndexSet, spec: dict, c0: np.ndarray, h: float, nsteps: int, m: int,
                      t0: float = 0.0, order: str = "sym"):
    """c^{n+1} = exp(Omega^n) c^n with the 2-stage Gauss-Legendre Magnus exponent, Eq. (2stageMagnus):
    Omega^n = -(i/2) h (A_1 + A_2) - (sqrt(3)/12) h^2 [A_2, A_1], A_j = A(t^n + c_j h),
    c_{1,2} = 1/2 -+ sqrt(3)/6.  Written as exp(-i h H) with the Hermitian
    H = (A_1 + A_2)/2 - i (sqrt(3) h / 12) (A_2 A_1 - A_1 A_2), whose action takes four products;
    each exponential by lanczos_exp."""
    c = np.array(c0, dtype=np.complex128)
    t = t0
    g = np.sqrt(3.0) * h / 12.0
    for _ in range(nsteps):
        (r1, a1), (r2, a2) = (potential_terms(spec, t + cj * h) for cj in MAGNUS4_NODES)

        def H(v, r1=r1, a1=a1, r2=r2, a2=a2):
            u1 = apply(S, r1, a1, spec["L"], v, order)
            u2 = apply(S, r2, a2, spec["L"], v, order)
            comm = apply(S, r2, a2, spec["L"], u1, order) - apply(S, r1, a1, spec["L"], u2, order)
            return 0.5 * (u1 + u2) - 1j * g * comm

        c, _, _ = lanczos_exp(H, c, h, m)
        t += h
    return c, t


# --------------------------------------------------------------------------- #
# gradient of a final-time objective w.r.t. a piecewise-constant control       #
# --------------------------------------------------------------------------- #

def control_objective_dense(S: IndexSet, spec: dict, c0: np.ndarray, phi: np.ndarray, dt: float, nsub: int,
                            order: str = "sym"):
    """J = |<phi, psi(T)>|^2 with psi propagated by the exact exponentials of the midpoint rule,
    psi_n = exp(-i dt A(t_{n-1} + dt/2)) psi_{n-1} (Eq. (expMPR) with the matrix exponential done
    exactly by scipy's expm on the dense A; tiny sets only).  Returns (J, a, states)."""
    import scipy.linalg
    psi = np.array(c0, dtype=np.complex128)
    states = [psi]
    for n in range(nsub):
        r, a = potential_terms(spec, (n + 0.5) * dt)
        A = dense_A(S, r, a, spec["L"], order)
        psi = scipy.linalg.expm(-1j * dt * A) @ psi
        states.append(psi)
    amp = np.vdot(phi, psi)
    return float(abs(amp) ** 2), amp, states


def control_gradient_dense(S: IndexSet, spec: dict, c0: np.ndarray, phi: np.ndarray, dt: float, nsub: int,
                           n_intervals: int, order: str = "sym"):
    """dJ/du_q for the control u(t) x_1 (piecewise constant on n_intervals equal intervals of [0, nsub dt]).

    J = |a|^2, a = <phi, psi_M>; with lambda_M = phi and lambda_{n-1} = U_n^H lambda_n,
    da/du_q = sum over sub-steps n inside interval q of lambda_n^H (dU_n/du) psi_{n-1}, where dU_n/du is
    the Frechet derivative of exp at -i dt A_n in the direction -i dt X_1 (scipy's expm_frechet), and
    dJ/du_q = 2 Re(conj(a) da/du_q)."""
    import scipy.linalg
    J, amp, states = control_objective_dense(S, spec, c0, phi, dt, nsub, order)
    X1 = dense_X(S, 0)
    lam = np.array(phi, dtype=np.complex128)
    grad_a = np.zeros(n_intervals, dtype=np.complex128)
    per = nsub // n_intervals
    for n in range(nsub, 0, -1):
        r, a = potential_terms(spec, (n - 0.5) * dt)
        A = dense_A(S, r, a, spec["L"], order)
        U, Lf = scipy.linalg.expm_frechet(-1j * dt * A, -1j * dt * X1)
        grad_a[(n - 1) // per] += np.vdot(lam, Lf @ states[n - 1])
        lam = U.conj().T @ lam
    return J, 2.0 * np.real(np.conj(amp) * grad_a)


def control_gradient_matfree(S: IndexSet, spec: dict, c0: np.ndarray, phi: np.ndarray, dt: float, nsub: int,
                             n_intervals: int, m: int, order: str = "sym", gl_nodes: int = 8):
    """The gradient of control_gradient_dense without any matrix: every exponential is an m-step
    Lanczos exponential (lanczos_exp; the caller takes m and dt where it has converged) and the
    Frechet derivative of exp at -i dt A_n in the direction -i dt X_1 is applied through its integral
        lambda^H L psi = int_0^1 (e^{+i s dt A} lambda)^H (-i dt X_1) (e^{-i (1 - s) dt A} psi) ds,
    evaluated by Gauss-Legendre quadrature in s (the integrand is an entire function of s).  States
    psi_n are propagated forward, lambda_{n-1} = exp(+i dt A_n) lambda_n backward.  Returns (J, dJ/du)."""
    x, w = np.polynomial.legendre.leggauss(gl_nodes)
    s_nodes, s_weights = 0.5 * (x + 1.0), 0.5 * w
    psi = np.array(c0, dtype=np.complex128)
    states = [psi]
    for n in range(nsub):
        r, a = potential_terms(spec, (n + 0.5) * dt)
        psi = lanczos_exp(lambda v: apply(S, r, a, spec["L"], v, order), psi, dt, m)[0]
        states.append(psi)
    amp = np.vdot(phi, psi)
    lam = np.array(phi, dtype=np.complex128)
    grad_a = np.zeros(n_intervals, dtype=np.complex128)
    per = nsub // n_intervals
    for n in range(nsub, 0, -1):
        r, a = potential_terms(spec, (n - 0.5) * dt)
        Av = lambda v: apply(S, r, a, spec["L"], v, order)
        term = 0.0j
        for s, ws in zip(s_nodes, s_weights):
            right = lanczos_exp(Av, states[n - 1], (1.0 - s) * dt, m)[0]      # e^{-i (1-s) dt A} psi
            left = lanczos_exp(Av, lam, -s * dt, m)[0]                        # e^{+i s dt A} lambda
            term += ws * np.vdot(left, -1j * dt * direct_op(S, 0, right))
        grad_a[(n - 1) // per] += term
        lam = lanczos_exp(Av, lam, -dt, m)[0]                                 # U_n^H lambda = e^{+i dt A} lambda
    return float(abs(amp) ** 2), 2.0 * np.real(np.conj(amp) * grad_a)
