"""Pins of the oracle to facts other than itself (paper values, closed forms, library routines,
brute force).  CPU only."""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.special

from paper_1403_3511_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- #
# index sets                                                                   #
# --------------------------------------------------------------------------- #

def piltz_sum(N, B):
    """sum_{n <= B} d_N(n), d_N the N-fold divisor function built by Dirichlet convolution
    d_N = d_{N-1} * 1 (a divisor sieve), which counts {m in Z_{>=1}^N : prod m <= B} = |K_N(B)|."""
    d = np.ones(B + 1, dtype=np.int64)
    d[0] = 0
    for _ in range(N - 1):
        nd = np.zeros(B + 1, dtype=np.int64)
        for m in range(1, B + 1):
            nd[m::m] += d[1: B // m + 1]
        d = nd
    return int(d[1:].sum())


@pytest.mark.parametrize("N,B", [(1, 17), (2, 32), (3, 100), (4, 512), (6, 64), (10, 24)])
def test_count_equals_piltz_divisor_sum(oracle, N, B):
    assert oracle.hc_count(N, B) == piltz_sum(N, B)
    assert oracle.IndexSet.hyperbolic(N, B).size == piltz_sum(N, B)


def test_known_sizes(oracle):
    # sizes used by the workloads (Piltz sums, checked by the sieve above for the small ones)
    assert oracle.hc_count(2, 32) == 119
    assert oracle.hc_count(4, 512) == 37270
    assert piltz_sum(4, 512) == 37270


@pytest.mark.parametrize("N,B", [(2, 20), (3, 30), (4, 16)])
def test_enumeration_is_box_filter_in_lex_order(oracle, N, B):
    """Brute force: every k in the box [0, B-1]^N with prod(1 + k_l) <= B, sorted lexicographically."""
    S = oracle.IndexSet.hyperbolic(N, B)
    grids = np.meshgrid(*[np.arange(B)] * N, indexing="ij")
    box = np.stack([g.ravel() for g in grids], axis=1)
    keep = box[np.prod(1 + box, axis=1) <= B]
    assert np.array_equal(S.k, keep)              # meshgrid 'ij' ravel is lexicographic, last fastest
    for i in range(0, S.size, max(1, S.size // 50)):
        assert S.rank(S.k[i]) == i
    assert S.rank(np.full(N, B)) == -1


def test_downward_closed(oracle):
    """Sec. 1.2: k in K with k_l > 0 implies k - e_l in K."""
    S = oracle.IndexSet.hyperbolic(3, 60)
    for k in S.k:
        for l in range(3):
            if k[l] > 0:
                km = k.copy()
                km[l] -= 1
                assert S.rank(km) >= 0


# --------------------------------------------------------------------------- #
# Hermite basis and coordinate matrices                                        #
# --------------------------------------------------------------------------- #

def hermite_explicit(k, x):
    """phi_k(x) = pi^{-1/4} (2^k k!)^{-1/2} H_k(x) e^{-x^2/2}, the explicit form of Sec. 1.1 (scipy's H_k)."""
    return math.pi ** -0.25 / math.sqrt(2.0 ** k * math.factorial(k)) * scipy.special.eval_hermite(k, x) * np.exp(-x * x / 2)


def test_recurrence_matches_explicit_hermite_functions(oracle):
    x = np.linspace(-4, 4, 17)
    h = oracle.hermite_functions_scaled(12, x) * np.exp(-x * x / 2)
    for k in range(13):
        assert np.allclose(h[k], hermite_explicit(k, x), atol=1e-13)


def test_coordinate_matrix_is_position_operator(oracle):
    """(X^{(l)})_{jk} = (phi_j, x_l phi_k) on the full set, integrated by scipy's Gauss-Hermite
    rule with the explicit Hermite functions (exact: the integrand is a polynomial of low degree)."""
    S = oracle.IndexSet.full(2, 6)
    xi, w = scipy.special.roots_hermite(40)
    phi = np.array([hermite_explicit(k, xi) * np.exp(xi * xi / 2) for k in range(7)])
    M1 = np.einsum("m,jm,km->jk", w * xi, phi, phi)     # (phi_j, x phi_k)
    M0 = np.einsum("m,jm,km->jk", w, phi, phi)          # (phi_j, phi_k) = delta
    assert np.allclose(M0, np.eye(7), atol=1e-13)
    for l in range(2):
        X = oracle.dense_X(S, l)
        ref = np.zeros_like(X)
        for a, ka in enumerate(S.k):
            for b, kb in enumerate(S.k):
                other = [i for i in range(2) if i != l][0]
                ref[a, b] = M1[ka[l], kb[l]] * M0[ka[other], kb[other]]
        assert np.allclose(X, ref, atol=1e-13)


def test_direct_op_matches_dense_matrix(oracle):
    S = oracle.IndexSet.hyperbolic(3, 40)
    rng = np.random.default_rng(0)
    v = rng.standard_normal(S.size) + 1j * rng.standard_normal(S.size)
    for l in range(3):
        assert np.allclose(oracle.direct_op(S, l, v), oracle.dense_X(S, l) @ v, atol=1e-14)


# --------------------------------------------------------------------------- #
# Chebyshev interpolation of W (Sec. 1.3)                                      #
# --------------------------------------------------------------------------- #

def test_monomial_interpolation_is_exact(oracle):
    """x = L T1, x^2 = L^2 (T0 + T2)/2, x^3 = L^3 (3 T1 + T3)/4, x^4 = L^4 (3 T0 + 4 T2 + T4)/8."""
    L = 7.5
    exact = {1: [0, 1], 2: [0.5, 0, 0.5], 3: [0, 0.75, 0, 0.25], 4: [0.375, 0, 0.5, 0, 0.125]}
    for p, coefs in exact.items():
        u = oracle.cheb_nodes(p)
        got = oracle.cheb_coeffs_1d((L * u) ** p)
        assert np.allclose(got, np.array(coefs) * L ** p, rtol=0, atol=1e-14 * L ** p)


def test_cos_interpolant_tensor_equals_rank_two_form(oracle):
    """cos(a - b) = cos a cos b + sin a sin b, and tensor Chebyshev interpolation of a product is the
    product of the 1-D interpolants, so the 9x9 tensor interpolant equals the rank-2 form."""
    L, R = inputs.half_width(1024), 8
    u = oracle.cheb_nodes(R)
    T = oracle.cheb_coeffs_2d(np.cos(L * u[:, None] - L * u[None, :]))
    c = oracle.cheb_coeffs_1d(np.cos(L * u))
    s = oracle.cheb_coeffs_1d(np.sin(L * u))
    assert np.allclose(T, np.outer(c, c) + np.outer(s, s), atol=1e-13)


def test_time_dependent_interpolant_by_angle_addition(oracle):
    """A potential whose shape changes with t, beta cos(x_a - x_b + omega t) + beta/2 cos(x_1/4 + omega t),
    is interpolated anew at every t (the time-propagation algorithm of Sec. 2.2, step (1)).  By
    cos(d + th) = cos d cos th - sin d sin th, cos(a - b) = cos a cos b + sin a sin b and
    sin(a - b) = sin a cos b - cos a sin b, and since tensor interpolation of a product is the product
    of the 1-D interpolants, its coefficients at each t follow from numpy's 1-D interpolants at the
    Chebyshev points of the first kind."""
    N, R, L, beta, omega = 3, 8, inputs.half_width(60), 0.2, 2.0
    spec = dict(N=N, L=L, potential=inputs.drifting_cos_chain(N, beta, omega, R))
    cheb = np.polynomial.chebyshev.chebinterpolate
    ca, sa = cheb(lambda u: np.cos(L * u), R), cheb(lambda u: np.sin(L * u), R)
    cq, sq = cheb(lambda u: np.cos(0.25 * L * u), R), cheb(lambda u: np.sin(0.25 * L * u), R)
    cos_d, sin_d = np.outer(ca, ca) + np.outer(sa, sa), np.outer(sa, ca) - np.outer(ca, sa)
    for t in (0.0, 0.37, 1.9):
        th = omega * t
        want = np.zeros((R + 1,) * N)
        pair = beta * (math.cos(th) * cos_d - math.sin(th) * sin_d)
        want[:, :, 0] += pair                                      # axes (0, 1), r_2 = 0
        want[0, :, :] += pair                                      # axes (1, 2), r_0 = 0
        want[:, 0, 0] += 0.5 * beta * (math.cos(th) * cq - math.sin(th) * sq)
        r, a = oracle.potential_terms(spec, t)
        got = np.zeros_like(want)
        for rr, aa in zip(r.tolist(), a.tolist()):
            got[tuple(rr)] += aa
        assert np.abs(got - want).max() <= 1e-13, (t, np.abs(got - want).max())


def test_potential_terms_henon_heiles(oracle):
    """lam x1^2 x2 - lam/3 x2^3 in Chebyshev form: x1^2 x2 = L^3/2 (T0 + T2)(u1) T1(u2), x2^3 = L^3/4 (3T1 + T3)(u2)."""
    spec = inputs.workload("hh2_b32")
    L, lam = spec["L"], 0.111
    r, a = oracle.potential_terms(spec, 0.0)
    got = {tuple(x): y for x, y in zip(r.tolist(), a.tolist()) if abs(y) > 1e-12}
    want = {(0, 1): lam * L ** 3 / 2 - lam / 3 * 0.75 * L ** 3, (2, 1): lam * L ** 3 / 2, (0, 3): -lam / 3 * 0.25 * L ** 3}
    assert set(got) == set(want)
    for k in want:
        assert got[k] == pytest.approx(want[k], rel=1e-13)


def test_modulations(oracle):
    assert oracle.modulation({"kind": "cos", "omega": 2.0, "phase": 0.5}, 0.3) == pytest.approx(math.cos(1.1))
    assert oracle.modulation({"kind": "sin2", "omega": 1.0}, 0.7) == pytest.approx(math.sin(0.7) ** 2)
    m = {"kind": "pwconst", "values": [1.0, 2.0, 3.0, 4.0], "t0": 0.0, "t1": 2.0}
    assert [oracle.modulation(m, t) for t in (0.0, 0.49, 0.5, 1.2, 1.99, 2.0)] == [1, 1, 2, 3, 4, 4]


# --------------------------------------------------------------------------- #
# the operator                                                                 #
# --------------------------------------------------------------------------- #

def random_terms(rng, N, nterms, rmax):
    r = rng.integers(0, rmax + 1, size=(nterms, N)).astype(np.int32)
    return r, rng.standard_normal(nterms)


@pytest.mark.parametrize("N,B", [(2, 24), (3, 30), (4, 20)])
@pytest.mark.parametrize("order", ["sym", "eq", "alg"])
def test_fast_algorithm_matches_dense_polynomial(oracle, N, B, order):
    """The literal stencil fast algorithm (C) against dense matrix polynomials of X_K (numpy)."""
    rng = np.random.default_rng(N * 100 + B)
    S = oracle.IndexSet.hyperbolic(N, B)
    r, a = random_terms(rng, N, 6, 3)
    L = 5.0
    v = rng.standard_normal(S.size) + 1j * rng.standard_normal(S.size)
    W = oracle.dense_W(S, r, a, L, order)
    got = oracle.fast_algorithm(S, r, a, L, v, order)
    assert np.allclose(got, W @ v, atol=1e-12 * np.abs(W @ v).max())


def test_symmetric_ordering(oracle):
    """With the symmetrised factor order A is exactly symmetric; the two literal orders are not on a
    reduced set (the coordinate matrices of different axes do not commute there)."""
    S = oracle.IndexSet.hyperbolic(2, 32)
    spec = inputs.workload("hh2_b32")
    r, a = oracle.potential_terms(spec, 0.0)
    Asym = oracle.dense_A(S, r, a, spec["L"], "sym")
    assert np.abs(Asym - Asym.T).max() <= 1e-13 * np.abs(Asym).max()
    for order in ("eq", "alg"):
        Ao = oracle.dense_A(S, r, a, spec["L"], order)
        assert np.abs(Ao - Ao.T).max() > 1e-3
    X1, X2 = oracle.dense_X(S, 0), oracle.dense_X(S, 1)
    assert np.abs(X1 @ X2 - X2 @ X1).max() > 0.1


def test_orders_agree_on_full_set(oracle):
    """Sec. 4.2: on K_full the factor order is arbitrary."""
    S = oracle.IndexSet.full(2, 7)
    rng = np.random.default_rng(3)
    r, a = random_terms(rng, 2, 5, 3)
    v = rng.standard_normal(S.size) + 0j
    eq = oracle.fast_algorithm(S, r, a, 4.0, v, "eq")
    alg = oracle.fast_algorithm(S, r, a, 4.0, v, "alg")
    assert np.allclose(eq, alg, atol=1e-12)


@pytest.mark.parametrize("N,K,R", [(1, 12, 5), (2, 6, 3), (3, 4, 2)])
def test_lemma1_full_set_insertion_equals_gh_quadrature(oracle, N, K, R):
    """Lemma 1 (Sec. 4.2): on K_full(K), inserting X_full into W^pol equals the (K+1)-point product
    Gauss-Hermite assembly, entrywise (nodes and weights from numpy's hermgauss)."""
    S = oracle.IndexSet.full(N, K)
    rng = np.random.default_rng(K)
    grids = np.meshgrid(*[np.arange(R + 1)] * N, indexing="ij")
    r = np.stack([g.ravel() for g in grids], axis=1).astype(np.int32)
    a = rng.standard_normal(len(r))
    L = 6.0
    W = oracle.dense_W(S, r, a, L, "sym")
    G = oracle.gh_assembly(S, r, a, L, K)
    assert np.abs(W - G).max() <= 1e-12 * max(1.0, np.abs(W).max())


def test_reduced_set_interior_rows_equal_exact_galerkin(oracle):
    """On a reduced set, rows j with j + deg in K carry no reduction error (remark after Thm. 2) and,
    for K >> R, no quadrature error either (Sec. 5.2): they equal the exact Galerkin matrix of W^pol,
    computed by Gauss-Hermite quadrature with enough nodes to be exact."""
    N, B = 2, 40
    S = oracle.IndexSet.hyperbolic(N, B)
    spec = inputs.workload("hh2_b32")
    spec = dict(spec, B=B, L=inputs.half_width(B))
    r, a = oracle.potential_terms(spec, 0.0)
    W = oracle.dense_W(S, r, a, spec["L"], "sym")
    Gex = oracle.gh_assembly(S, r, a, spec["L"], B + 8)
    deg = 3
    interior = [i for i, k in enumerate(S.k) if (1 + k[0] + deg) * (1 + k[1] + deg) <= B]
    assert len(interior) > 10
    assert np.abs(W[interior] - Gex[interior]).max() <= 1e-12 * np.abs(W).max()
    assert np.abs(W - Gex).max() > 1e-6          # the boundary rows do differ, by design


def test_local_rows_equal_full_apply(oracle):
    rng = np.random.default_rng(5)
    for name, N, B in [("hh", 4, 200), ("cos", 3, 120)]:
        if name == "hh":
            spec = dict(N=N, B=B, L=inputs.half_width(B), potential=inputs.henon_heiles_chain(N, 0.111, (0.05, 1.0)))
        else:
            spec = dict(N=N, B=B, L=inputs.half_width(B), potential=inputs.cos_chain(N, 0.2, 8))
        S = oracle.IndexSet.hyperbolic(N, B)
        r, a = oracle.potential_terms(spec, 0.3)
        c = rng.standard_normal(S.size) + 1j * rng.standard_normal(S.size)
        full = oracle.apply(S, r, a, spec["L"], c)
        rows = inputs.sample_rows(S.size, 60)
        loc = oracle.apply_rows(S, B, r, a, spec["L"], c, rows)
        assert np.allclose(loc, full[rows], atol=1e-12 * np.abs(full).max())


# --------------------------------------------------------------------------- #
# spectra (closed forms)                                                       #
# --------------------------------------------------------------------------- #

def test_harmonic_oscillator_spectrum(oracle):
    """W = 0: A = D_K with eigenvalues sum_l (k_l + 1/2), Eq. (EigenfunctionRelation)."""
    S = oracle.IndexSet.hyperbolic(3, 50)
    A = oracle.dense_A(S, np.zeros((0, 3), np.int32), np.zeros(0), 10.0)
    ev = np.sort(np.linalg.eigvalsh(A))
    assert np.allclose(ev, np.sort(S.k.sum(axis=1) + 1.5), atol=1e-13)


def test_linear_potential_shifts_spectrum(oracle):
    """W = a x_1: H = HO shifted by -a/... completing the square gives E = |n| + N/2 - a^2/2 for the
    low states (exponentially small truncation error at large B)."""
    N, B, a = 2, 400, 0.7
    S = oracle.IndexSet.hyperbolic(N, B)
    spec = dict(N=N, B=B, L=inputs.half_width(B), potential=[{"coef": a, "powers": {0: 1}}])
    r, al = oracle.potential_terms(spec, 0.0)
    ev = np.sort(np.linalg.eigvalsh(oracle.dense_A(S, r, al, spec["L"])))
    want = np.sort([n1 + n2 + 1.0 - a * a / 2 for n1 in range(6) for n2 in range(6)])[:8]
    assert np.allclose(ev[:8], want, atol=1e-10)


def test_coupled_quadratic_spectrum(oracle):
    """V = 1/2 x^T M x (W = V - |x|^2/2, mixed terms through the symmetrised product): eigenvalues
    sum_i (n_i + 1/2) sqrt(mu_i(M)).  Needs the Sym ordering of the mixed term x_1 x_2."""
    N, B = 2, 600
    M = np.array([[1.3, 0.25], [0.25, 0.8]])
    S = oracle.IndexSet.hyperbolic(N, B)
    comps = [{"coef": 0.5 * (M[0, 0] - 1), "powers": {0: 2}}, {"coef": 0.5 * (M[1, 1] - 1), "powers": {1: 2}},
             {"coef": M[0, 1], "powers": {0: 1, 1: 1}}]
    spec = dict(N=N, B=B, L=inputs.half_width(B), potential=comps)
    r, al = oracle.potential_terms(spec, 0.0)
    ev = np.sort(np.linalg.eigvalsh(oracle.dense_A(S, r, al, spec["L"])))
    w = np.sqrt(np.linalg.eigvalsh(M))
    want = np.sort([(n1 + 0.5) * w[0] + (n2 + 0.5) * w[1] for n1 in range(8) for n2 in range(8)])[:6]
    assert np.allclose(ev[:6], want, atol=1e-9)


@pytest.mark.parametrize("scale", [0.8, 1.3])
def test_scaled_basis_spectra(oracle, scale):
    """The basis phi_k(S x) (Sec. 1.4) changes the matrix but not the operator: for V = |x|^2 / 2
    (W = 0) on N = 1 the lowest eigenvalues stay k + 1/2, and for the coupled quadratic V = x^T M x / 2
    on a 2-d hyperbolic cross they stay sum_i (n_i + 1/2) sqrt(mu_i(M)).  A wrong factor of D_K, a
    wrong sign or size of the (1/S^2 - S^2)/2 X^2 term, or W not evaluated at X / S moves them."""
    S1 = oracle.IndexSet.hyperbolic(1, 80)
    ev = np.sort(np.linalg.eigvalsh(oracle.dense_A(S1, np.zeros((0, 1), np.int32), np.zeros(0), 13.0, scale=scale)))
    assert np.allclose(ev[:8], np.arange(8) + 0.5, atol=1e-9), ev[:8]
    N, B = 2, 600
    M = np.array([[1.3, 0.25], [0.25, 0.8]])
    S = oracle.IndexSet.hyperbolic(N, B)
    comps = [{"coef": 0.5 * (M[0, 0] - 1), "powers": {0: 2}}, {"coef": 0.5 * (M[1, 1] - 1), "powers": {1: 2}},
             {"coef": M[0, 1], "powers": {0: 1, 1: 1}}]
    spec = dict(N=N, B=B, L=inputs.half_width(B), potential=comps)
    r, al = oracle.potential_terms(spec, 0.0)
    A = oracle.dense_A(S, r, al, spec["L"], scale=scale)
    ev = np.sort(np.linalg.eigvalsh(A))
    w = np.sqrt(np.linalg.eigvalsh(M))
    want = np.sort([(n1 + 0.5) * w[0] + (n2 + 0.5) * w[1] for n1 in range(8) for n2 in range(8)])[:6]
    assert np.allclose(ev[:6], want, atol=1e-8), (ev[:6], want)
    # the matrix-free product is the same matrix
    c = inputs.initial_vector({"init": {"kind": "gaussian", "seed": 4}}, S.k)
    assert np.abs(oracle.apply(S, r, al, spec["L"], c, scale=scale) - A @ c).max() <= 1e-11 * np.abs(A @ c).max()


def test_general_downward_closed_sets(oracle):
    """A total-degree set {|k|_1 <= 6} and a seeded random downward-closed set, given as lists: the
    matrix-free product equals the dense matrix built from the recurrence on the same set (both
    orders of the mixed term averaged), and for W = 0 it is D_K exactly."""
    for ks in (inputs.total_degree_set(3, 6), inputs.random_downward_closed_set(3, 60, seed=8)):
        S = oracle.IndexSet.from_list(ks)
        spec = dict(N=3, L=6.0, potential=inputs.henon_heiles_chain(3, 0.111, (0.05, 1.0)))
        r, al = oracle.potential_terms(spec, 0.3)
        c = inputs.initial_vector({"init": {"kind": "gaussian", "seed": 5}}, S.k)
        A = oracle.dense_A(S, r, al, spec["L"])
        assert np.abs(oracle.apply(S, r, al, spec["L"], c) - A @ c).max() <= 1e-12 * np.abs(A @ c).max()
        assert np.allclose(A, A.T, atol=1e-12)
        y0 = oracle.apply(S, np.zeros((0, 3), np.int32), np.zeros(0), spec["L"], c)
        assert np.array_equal(y0, oracle.diag(S) * c)


def test_matrix_free_adjoint_matches_dense(oracle):
    """The matrix-free FP64 adjoint gradient (Lanczos exponentials, Gauss-Legendre quadrature of the
    Frechet derivative) against the dense one (scipy's expm_frechet) on N = 2, B = 10, where m = |K|
    makes every Lanczos exponential exact.  A sign error in either exponential of the integrand, a
    missing dt, or lambda propagated the wrong way breaks it."""
    N, B = 2, 10
    S = oracle.IndexSet.hyperbolic(N, B)
    u = np.array([0.07, -0.05, 0.02, 0.09])
    T, substeps = 0.8, 2
    spec = dict(N=N, B=B, L=inputs.half_width(B), potential=inputs.control_quartic(u, T))
    c0 = inputs.initial_vector({"init": {"kind": "coherent", "q": [1.0, 0.0], "eps": 0.0, "seed": 0}}, S.k)
    phi = np.zeros(S.size, complex)
    phi[S.rank([1, 0])] = 1.0
    dt = T / (len(u) * substeps)
    J_d, g_d = oracle.control_gradient_dense(S, spec, c0, phi, dt, len(u) * substeps, len(u))
    J_m, g_m = oracle.control_gradient_matfree(S, spec, c0, phi, dt, len(u) * substeps, len(u), m=S.size)
    assert abs(J_m - J_d) <= 1e-12 * J_d
    assert np.abs(g_m - g_d).max() <= 1e-11 * np.abs(g_d).max(), (g_m, g_d)


# --------------------------------------------------------------------------- #
# paper tables                                                                 #
# --------------------------------------------------------------------------- #

def torsional_spec(N):
    """W = sum_l (1 - cos(x_l / 16)) with L = 16, R = 8 (Eq. (TorsionalPotential))."""
    comps = [{"coef": -1.0, "func": "cos_scaled", "axes": [l], "scale": 1 / 16.0, "R": 8} for l in range(N)]
    return dict(N=N, L=16.0, potential=comps)


@pytest.mark.parametrize("N,K", [(2, 25), (2, 50), (2, 75), (3, 25), (3, 50), (4, 25)])
def test_fig5_local_error_table(oracle, N, K):
    """Reproduces the printed E^quad v and E^red(v) of Fig. 5 (Sec. 6.1) to the printed digits."""
    gold = json.load(open(os.path.join(GOLDEN, "fig5_local_errors.json")))
    S = oracle.IndexSet.hyperbolic(N, K + 1)
    r, a = oracle.potential_terms(torsional_spec(N), 0.0)
    r = np.vstack([r, np.zeros((1, N), np.int32)])
    a = np.append(a, float(N))                       # the constant sum_l 1
    v = inputs.initial_vector({"init": {"kind": "beta_decay", "beta": 5.0}}, S.k).real
    fast = oracle.fast_algorithm(S, r, a, 16.0, v.astype(complex)).real
    G = oracle.gh_assembly(S, r, a, 16.0, K)            # GH(K): K + 1 nodes per axis
    Gex = oracle.gh_assembly(S, r, a, 16.0, K + 10)     # exact for this polynomial
    e_red = np.abs(fast - G @ v).max()
    e_quad = np.abs(Gex @ v - G @ v).max()
    i = gold["K"].index(K)
    assert e_red == pytest.approx(gold["E_red"][str(N)][i], rel=1.5e-3)
    assert e_quad == pytest.approx(gold["E_quad"][str(N)][i], rel=1.5e-3)


# --------------------------------------------------------------------------- #
# time integration                                                             #
# --------------------------------------------------------------------------- #

def test_lanczos_matches_dense_expm(oracle):
    """With m large enough, beta_0 V_m exp(-ihT_m) e_1 converges to exp(-ihA) c (scipy expm)."""
    N, B = 2, 30
    S = oracle.IndexSet.hyperbolic(N, B)
    spec = dict(inputs.workload("hh2_b32"), B=B, L=inputs.half_width(B))
    r, a = oracle.potential_terms(spec, 0.0)
    A = oracle.dense_A(S, r, a, spec["L"])
    c = inputs.initial_vector(spec, S.k)
    h = 0.05
    ref = scipy.linalg.expm(-1j * h * A) @ c
    got, al, be = oracle.lanczos_exp(lambda v: A @ v, c, h, 14)
    assert np.linalg.norm(got - ref) <= 1e-12
    got7, _, _ = oracle.lanczos_exp(lambda v: A @ v, c, h, 7)
    assert np.linalg.norm(got7 - ref) > 1e-14         # truncation error of m = 7 is visible


def test_lanczos_error_estimate_tracks_true_error(oracle):
    """The a-posteriori estimate |h| beta_m |e_m^T exp(-ihT_m) e_1| (Sec. 2.2: the residual of the
    Lanczos relation) against the true relative error from scipy's expm, over step sizes from the
    unresolved to the converged regime: an upper bound within a factor 2m wherever the error is
    above round-off, and once converged the ratio tends to m (the leading term of the error is
    h^m/m! times the product of the betas, that of the estimate h^m/(m-1)! times the same), monotone
    in h, and zero after an exact breakdown.  A dropped beta_m, a wrong component of exp(-ihT_m) e_1
    (first instead of last) or a missing h breaks the ratio."""
    N, B = 2, 30
    S = oracle.IndexSet.hyperbolic(N, B)
    spec = dict(inputs.workload("hh2_b32"), B=B, L=inputs.half_width(B))
    r, a = oracle.potential_terms(spec, 0.0)
    A = oracle.dense_A(S, r, a, spec["L"])
    c = inputs.initial_vector({"init": {"kind": "gaussian", "seed": 9}}, S.k)
    ests, m = [], 7
    for h in (0.3, 0.2, 0.1, 0.05, 0.02, 0.01):
        ref = scipy.linalg.expm(-1j * h * A) @ c
        got, _, _, est = oracle.lanczos_exp(lambda v: A @ v, c, h, m, estimate=True)
        err = np.linalg.norm(got - ref) / np.linalg.norm(c)
        ests.append(est)
        if err > 1e-12:
            assert 1.0 <= est / err <= 2 * m, (h, est, err)
        if h <= 0.02:
            assert abs(est / err - m) <= 0.05 * m, (h, est / err)
    assert all(x > y for x, y in zip(ests, ests[1:]))
    S3 = oracle.IndexSet.hyperbolic(3, 30)
    d = oracle.diag(S3)
    c3 = np.zeros(S3.size, complex)
    for lev in (1.5, 3.5, 6.5):
        c3[np.where(d == lev)[0]] = 1.0
    assert oracle.lanczos_exp(lambda v: d * v, c3, 0.3, 7, estimate=True)[3] == 0.0


def test_lanczos_exact_on_few_levels(oracle):
    """W = 0, c supported on 3 distinct levels of D: Lanczos terminates (breakdown) and the step equals
    the exact c_k exp(-i (|k| + N/2) h)."""
    S = oracle.IndexSet.hyperbolic(3, 30)
    d = oracle.diag(S)
    c = np.zeros(S.size, complex)
    for lev in (1.5, 3.5, 6.5):
        c[np.where(d == lev)[0]] = 0.3 + 0.1j
    h = 0.37
    got, al, _ = oracle.lanczos_exp(lambda v: d * v, c, h, 7)
    assert len(al) == 3
    assert np.allclose(got, np.exp(-1j * d * h) * c, atol=1e-13)


def test_expmpr_norm_conservation_and_order(oracle):
    """The exponential midpoint rule (Eq. (expMPR)) conserves the norm and converges with order 2
    for a time-dependent potential (dipole cos(t) x_1)."""
    N, B = 2, 24
    S = oracle.IndexSet.hyperbolic(N, B)
    spec = dict(N=N, B=B, L=inputs.half_width(B),
                potential=inputs.henon_heiles_chain(N, 0.111, dipole=(0.5, 3.0)),
                init={"kind": "coherent", "q": [1.0, 0.5], "eps": 0.0, "seed": 0})
    c0 = inputs.initial_vector(spec, S.k)
    T = 0.4

    def run(h, m):
        c, _ = oracle.expmpr_propagate(S, spec, c0, h, int(round(T / h)), m)
        return c

    ref = run(T / 640, 12)
    errs = [np.linalg.norm(run(T / n, 12) - ref) for n in (10, 20, 40)]
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.8 < s < 2.3 for s in slopes), slopes
    c = run(T / 20, 7)
    assert abs(np.linalg.norm(c) - 1.0) < 1e-13


def test_coherent_state_closed_form(oracle):
    """The closed-form Hermite coefficients of the Gaussian wave packet equal its projections
    (psi_0, phi_k) by Gauss-Hermite quadrature with the explicit Hermite functions."""
    q = 0.8
    xi, w = scipy.special.roots_hermite(80)
    psi = math.pi ** -0.25 * np.exp(-(xi - q) ** 2 / 2) * np.exp(xi * xi)   # divided by the weight e^{-x^2}
    proj = [np.sum(w * psi * hermite_explicit(k, xi)) for k in range(15)]
    got = inputs.coherent_state(np.arange(15)[:, None], [q]).real
    assert np.allclose(got, proj, atol=1e-13)


def test_control_gradient_matches_central_differences(oracle):
    """The FP64 adjoint gradient equals central finite differences of the objective (h = 1e-6)."""
    N, B = 2, 10
    S = oracle.IndexSet.hyperbolic(N, B)
    u = np.array([0.07, -0.05, 0.02, 0.09])
    spec = dict(N=N, B=B, L=inputs.half_width(B), potential=inputs.control_quartic(u, 0.8))
    c0 = inputs.initial_vector({"init": {"kind": "coherent", "q": [1.0, 0.0], "eps": 0.0, "seed": 0}}, S.k)
    phi = np.zeros(S.size, complex)
    phi[S.rank([1, 0])] = 1.0
    dt, nsub = 0.1, 8
    J, g = oracle.control_gradient_dense(S, spec, c0, phi, dt, nsub, len(u))
    h = 1e-6
    for q in range(len(u)):
        up, um = u.copy(), u.copy()
        up[q] += h
        um[q] -= h
        Jp, _, _ = oracle.control_objective_dense(S, dict(spec, potential=inputs.control_quartic(up, 0.8)), c0, phi, dt, nsub)
        Jm, _, _ = oracle.control_objective_dense(S, dict(spec, potential=inputs.control_quartic(um, 0.8)), c0, phi, dt, nsub)
        fd = (Jp - Jm) / (2 * h)
        assert abs(g[q] - fd) <= 1e-7 * max(abs(fd), 1e-3), (q, g[q], fd)
    assert np.abs(g).max() > 1e-4


def _time_dependent_hh2():
    N, B = 2, 12
    return dict(N=N, B=B, L=inputs.half_width(B),
                potential=inputs.henon_heiles_chain(N, 0.2) + [{"coef": 0.8, "powers": {0: 1},
                                                                "mod": {"kind": "sin2", "omega": 2.0}}])


def _drifting_cos2():
    """cos(x_1 - x_2 + 2t) chain with cos(x_1/4 + 2t): a potential whose interpolant changes shape with t."""
    N, B = 2, 12
    return dict(N=N, B=B, L=inputs.half_width(B), potential=inputs.drifting_cos_chain(N, 0.6, 2.0))


@pytest.mark.parametrize("make_spec", [_time_dependent_hh2, _drifting_cos2])
def test_magnus4_is_order_four_and_midpoint_order_two(oracle, make_spec):
    """Eq. (2stageMagnus) has order 4 and Eq. (expMPR) order 2 (Sec. 2.1): with exact exponentials
    (m = |K|), against scipy's DOP853 solution of i c' = A(t) c with the same dense matrices, halving h
    divides the error by 16 and by 4.  Also when the potential is re-interpolated at every evaluation
    time (a shape that drifts with t)."""
    from scipy.integrate import solve_ivp
    spec = make_spec()
    S = oracle.IndexSet.hyperbolic(spec["N"], spec["B"])
    c0 = inputs.initial_vector({"init": {"kind": "coherent", "q": [0.7, -0.4], "eps": 0.0, "seed": 0}}, S.k)

    def rhs(t, y):
        r, a = oracle.potential_terms(spec, t)
        return -1j * (oracle.dense_A(S, r, a, spec["L"]) @ y)

    ref = solve_ivp(rhs, (0.0, 1.0), c0, method="DOP853", rtol=1e-13, atol=1e-15).y[:, -1]
    err = {}
    for h in (0.2, 0.1):
        n = round(1.0 / h)
        err["m4", h] = np.linalg.norm(oracle.magnus4_propagate(S, spec, c0, h, n, S.size)[0] - ref)
        err["mpr", h] = np.linalg.norm(oracle.expmpr_propagate(S, spec, c0, h, n, S.size)[0] - ref)
    assert 14.0 < err["m4", 0.2] / err["m4", 0.1] < 18.0, err
    assert 3.6 < err["mpr", 0.2] / err["mpr", 0.1] < 4.4, err
    assert err["m4", 0.1] < 1e-2 * err["mpr", 0.1]


def test_magnus4_without_time_dependence_is_the_midpoint_rule(oracle):
    """For a time-independent A the commutator in Eq. (2stageMagnus) vanishes and Omega = -i h A."""
    spec = inputs.workload("hh2_b32")
    S = oracle.IndexSet.hyperbolic(spec["N"], spec["B"])
    c0 = inputs.initial_vector(spec, S.k)
    a, _ = oracle.magnus4_propagate(S, spec, c0, 0.05, 4, 7)
    b, _ = oracle.expmpr_propagate(S, spec, c0, 0.05, 4, 7)
    assert np.abs(a - b).max() <= 1e-13


def test_time_integration_table(oracle):
    """The time-integration table of Sec. 6.3 for N = 2, K = 40, m = 7, against the exact-Galerkin
    reference.  Where the time discretisation dominates (expMPR, h >= 1/40; the 2-stage Magnus method,
    h = 1/10) the printed errors are reproduced to 2 % and 8 %; the plateau (the reduction error of
    the fast algorithm, which the printed potential leaves under-determined) to a factor 1.6."""
    gold = json.load(open(os.path.join(GOLDEN, "fig10_time_integration.json")))
    rows = {(r["N"], r["m"], r["K"], r["scheme"]): r["err"] for r in gold["rows"]}
    spec = inputs.time_integration_workload(2, 40)
    S = oracle.IndexSet.hyperbolic(2, spec["B"])
    c0 = inputs.initial_vector(spec, S.k)
    ref = oracle.galerkin_reference(S, spec, c0, 1.0)
    mpr = rows[2, 7, 40, "expmpr"]
    for i, h in enumerate(gold["h"][:3]):
        c, _ = oracle.expmpr_propagate(S, spec, c0, h, round(1.0 / h), 7)
        assert abs(np.abs(c - ref).max() / mpr[i] - 1.0) < 0.02, (h, np.abs(c - ref).max(), mpr[i])
    c, _ = oracle.magnus4_propagate(S, spec, c0, 0.1, 10, 7)
    assert abs(np.abs(c - ref).max() / rows[2, 7, 40, "magnus4"][0] - 1.0) < 0.08
    c, _ = oracle.magnus4_propagate(S, spec, c0, 0.025, 40, 7)
    plateau = np.abs(c - ref).max()
    assert 1.0 < plateau / rows[2, 7, 40, "magnus4"][-1] < 1.6


# --------------------------------------------------------------------------- #
# perturbed Lanczos (Sec. 6.2)                                                 #
# --------------------------------------------------------------------------- #

def test_fig8_perturbed_lanczos_soft_pin(oracle):
    """Sec. 6.2, Fig. 8: the error of an m = 5 Lanczos step when the fast algorithm replaces the
    exact Galerkin product, read with the unperturbed A = D_K + (exact Galerkin matrix of the
    interpolated W), v_k = prod max(k_l, 1)^-3 normalised, and max-abs (the norm that reproduces
    Fig. 5).  The N = 4 row is reproduced (0.2 %), N = 3 to 4 %, the N = 2 rows within a factor 1.6
    (a soft pin); linear in h (each halving of h halves the error to 8 %; the printed ratios run from
    1.99 to 2.105); smaller for larger K at N = 2 and larger for larger N at K = 40, as printed."""
    gold = json.load(open(os.path.join(GOLDEN, "fig8_perturbed_lanczos.json")))
    m, beta = gold["m"], gold["beta"]
    first = {}
    for row in gold["rows"]:
        N, K = row["N"], row["K"]
        S = oracle.IndexSet.hyperbolic(N, K + 1)
        r, a = oracle.potential_terms(torsional_spec(N), 0.0)
        r = np.vstack([r, np.zeros((1, N), np.int32)])
        a = np.append(a, float(N))
        v = inputs.initial_vector({"init": {"kind": "beta_decay", "beta": beta}}, S.k)
        d = oracle.diag(S)
        A = np.diag(d) + oracle.gh_assembly(S, r, a, 16.0, K + 10)      # exact for this polynomial
        errs = []
        for h in gold["h"]:
            up, _, _ = oracle.lanczos_exp(lambda x: A @ x, v, h, m)
            pe, _, _ = oracle.lanczos_exp(lambda x: d * x + oracle.fast_algorithm(S, r, a, 16.0, x), v, h, m)
            errs.append(np.abs(up - pe).max())
        # N = 4 reproduces the printed row to 0.2 %, N = 3 to 4 %; the N = 2 rows come out a constant
        # factor 1.10 ... 1.41 above theirs
        tol = {4: 1.005, 3: 1.05}.get(N, 1.6)
        for e, p in zip(errs, row["err"]):
            assert p / tol <= e <= p * tol, (N, K, e, p)
        for e0, e1 in zip(errs, errs[1:]):
            assert e0 / e1 == pytest.approx(2.0, rel=0.08)     # printed ratios: 1.99 ... 2.105
        first[(N, K)] = errs[0]
    assert first[(2, 10)] > first[(2, 20)] > first[(2, 30)] > first[(2, 40)]
    assert first[(2, 40)] < first[(3, 40)] < first[(4, 40)]


def test_fig9_lanczos_error_table_soft_pin(oracle):
    """Sec. 6.2, Fig. 9 (h = 1/10): the unperturbed Lanczos error (against exp(-ihA) v by scipy's
    expm) and the perturbation error, with the readings of the Fig. 8 pin.  A soft pin: every
    printed cell within a factor 2.5 (the m = 9, K = 10 entry is 1e-13, rounding level), and the
    structure the paper draws from the table: at N = 2 the unperturbed error falls with m and rises
    with K, the perturbation error falls with K and hardly depends on m (m >= 5: within 3 %)."""
    gold = json.load(open(os.path.join(GOLDEN, "fig9_lanczos_errors.json")))
    h = gold["h"]
    got = {}
    for row in gold["rows"]:
        N, m = row["N"], row["m"]
        un, pe = [], []
        for K in gold["K"]:
            S = oracle.IndexSet.hyperbolic(N, K + 1)
            r, a = oracle.potential_terms(torsional_spec(N), 0.0)
            r = np.vstack([r, np.zeros((1, N), np.int32)])
            a = np.append(a, float(N))
            v = inputs.initial_vector({"init": {"kind": "beta_decay", "beta": gold["beta"]}}, S.k)
            d = oracle.diag(S)
            A = np.diag(d) + oracle.gh_assembly(S, r, a, 16.0, K + 10)
            up, _, _ = oracle.lanczos_exp(lambda x: A @ x, v, h, m)
            pf, _, _ = oracle.lanczos_exp(lambda x: d * x + oracle.fast_algorithm(S, r, a, 16.0, x), v, h, m)
            un.append(np.abs(up - scipy.linalg.expm(-1j * h * A) @ v).max())
            pe.append(np.abs(up - pf).max())
        for e, p in zip(un + pe, row["unperturbed"] + row["perturbation"]):
            assert p / 2.5 <= e <= p * 2.5, (N, m, e, p)
        got[(N, m)] = (un, pe)
    for mlo, mhi in ((3, 5), (5, 7), (7, 9)):
        assert all(x > y for x, y in zip(got[(2, mlo)][0], got[(2, mhi)][0]))
    for m in (3, 5, 7, 9):
        un, pe = got[(2, m)]
        assert un == sorted(un) and pe == sorted(pe, reverse=True)
    for m in (7, 9):
        assert np.allclose(got[(2, m)][1], got[(2, 5)][1], rtol=0.03)
