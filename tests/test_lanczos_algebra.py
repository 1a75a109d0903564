"""The Lanczos recurrence the complex64/complex128 step kernels implement for m <= 8 (one
Gram-Schmidt sweep per Lanczos vector: the second pass of v_k lagged into the sweep that makes the
first pass of v_{k+1}, the first-pass coefficients taken from the three-term relation, only
<v_k, A v_k> measured from the product), restated here in numpy from the kernels' documented
formulas and checked against the oracle's classical Gram-Schmidt applied twice (Sec. 2.2): the same
T_m and the same exponential, in FP64 to rounding.  No GPU: this pins the algebra the sweep kernel
is written from, the GPU tests pin the kernels."""
import numpy as np
import pytest


def one_sweep_lanczos(A, c, m):
    """alpha, beta (beta[k] after vector k) and V of the one-sweep recurrence."""
    n = c.shape[0]
    U = c / np.linalg.norm(c)          # u_0: first-pass direction (unit norm)
    V = np.zeros((m, n), complex)
    p = np.zeros(0, complex)           # p_j = <v_j, u_k>
    nu = 1.0                           # ||u_k - sum_j p_j v_j||
    al, be = np.zeros(m), np.zeros(m)
    for k in range(m):
        z = A @ U                                       # the product launch
        r = np.vdot(U, z)                               # its Rayleigh quotient
        q = np.zeros(k, complex)                        # q_j = <A v_j, u_k> from the relation
        for j in range(k):
            q[j] = al[j] * p[j] + (be[j - 1] * p[j - 1] if j > 0 else 0.0) + be[j] * (p[j + 1] if j + 1 < k else nu)
        ck = (r - np.vdot(p, q)) / nu ** 2
        vk = (U - p @ V[:k]) / nu                        # the sweep
        w = (z - q @ V[:k]) / nu - ck * vk
        V[k] = vk
        d = V[:k + 1].conj() @ w
        nw = np.linalg.norm(w)
        hk = ck - (p[k - 1] * be[k - 1] / nu if k > 0 else 0.0)
        al[k] = (hk + d[k]).real
        p = d / nw
        nu = np.sqrt(max(1.0 - np.vdot(p, p).real, 0.0))
        be[k] = nw * nu
        U = w / nw
    return al, be, V


@pytest.mark.parametrize("seed,m", [(1, 7), (2, 8), (3, 4)])
def test_one_sweep_recurrence_matches_oracle_lanczos(oracle, seed, m):
    rng = np.random.default_rng(seed)
    n = 300
    Q = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))[0]
    lam = np.concatenate([rng.uniform(0.0, 3e4, n - 4), [0.5, 1.5, 2.9e4, 3e4]])
    A = (Q * lam) @ Q.conj().T
    A = (A + A.conj().T) / 2
    c = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    h = 1e-5
    ref, al_ref, be_ref = oracle.lanczos_exp(lambda v: A @ v, c, h, m)
    al, be, V = one_sweep_lanczos(A, c, m)
    assert np.abs(al - np.asarray(al_ref)).max() <= 1e-13 * np.abs(al_ref).max()
    assert np.abs(be[: m - 1] - np.asarray(be_ref)[: m - 1]).max() <= 1e-13 * np.abs(be_ref).max()
    assert np.abs(V.conj() @ V.T - np.eye(m)).max() <= 1e-13
    T = np.diag(al) + np.diag(be[: m - 1], 1) + np.diag(be[: m - 1], -1)
    lam_t, Qt = np.linalg.eigh(T)
    y = np.linalg.norm(c) * (V.T @ (Qt @ (np.exp(-1j * h * lam_t) * Qt[0].conj())))
    assert np.linalg.norm(y - ref) <= 1e-12 * np.linalg.norm(ref)
