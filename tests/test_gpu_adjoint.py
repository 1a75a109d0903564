"""GPU parity of the adjoint gradient (hx_adjoint_grad) with respect to a piecewise-constant control."""
import numpy as np
import pytest

from paper_1403_3511_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_3511_gb300 import build
    build.build()
    from paper_1403_3511_gb300 import hx as _hx
    return _hx


def fixed_terms(hx, L):
    """The control problem's fixed part 0.1 x_1^2 x_2^2 (the control term is added by the library)."""
    spec = dict(L=L, potential=[{"coef": 0.1, "powers": {0: 2, 1: 2}}])
    return hx.terms_from_spec(spec)


def test_tiny_gradient_matches_oracle_adjoint(hx, oracle):
    """N=2, B=10 (|K| = 27): with m = 27 the Lanczos exponential is exact, so the GPU gradient is the
    gradient of the exact midpoint-rule propagator, which the oracle computes densely (expm_frechet)."""
    N, B = 2, 10
    L = inputs.half_width(B)
    S = oracle.IndexSet.hyperbolic(N, B)
    u = np.array([0.07, -0.05, 0.02, 0.09])
    T, substeps = 0.8, 2
    spec = dict(N=N, B=B, L=L, potential=inputs.control_quartic(u, T))
    c0 = inputs.initial_vector({"init": {"kind": "coherent", "q": [1.0, 0.0], "eps": 0.0, "seed": 0}}, S.k)
    phi = np.zeros(S.size, complex)
    phi[S.rank([1, 0])] = 1.0
    dt = T / (len(u) * substeps)
    J_ref, g_ref = oracle.control_gradient_dense(S, spec, c0, phi, dt, len(u) * substeps, len(u))
    s = hx.hx_indexset_create(N, B)
    try:
        cd = torch.from_numpy(c0).to("cuda")
        pd = torch.from_numpy(phi).to("cuda")
        J, g = hx.hx_adjoint_grad(s, L, fixed_terms(hx, L), 0, u, 0.0, T, substeps, cd, pd, m=S.size)
    finally:
        hx.hx_indexset_destroy(s)
    assert abs(J - J_ref) <= 1e-12 * abs(J_ref)
    assert np.abs(g - g_ref).max() <= 1e-10 * np.abs(g_ref).max(), (g, g_ref)


def test_control_problem_gradient_matches_central_differences(hx):
    """The N=4, B=512 control problem (200 intervals x 10 sub-steps, T = 10): adjoint gradient against
    central differences of the same FP64 objective at sampled intervals.

    J comes out of 2000 Lanczos steps and carries rounding of about eps = 1e-13 * J, so a central
    difference with step h has an error up to 2 eps / h on top of its O(h^2) truncation: with h = 1e-6
    that is 6e-8, comparable to the smallest gradient entries.  The largest entry is checked with
    h = 1e-6; the smallest with the Richardson-extrapolated difference (4 D(h/2) - D(h)) / 3, h = 2e-4,
    whose truncation is O(h^4) and whose rounding error is at most 3 eps / h."""
    spec = inputs.workload("ctrl4_b512")
    N, B, L = spec["N"], spec["B"], spec["L"]
    u = np.array(spec["u"])
    s = hx.hx_indexset_create(N, B)
    try:
        k = hx.hx_indexset_export(s, N)
        c0 = torch.from_numpy(inputs.initial_vector(spec, k)).to("cuda")
        phi_h = np.zeros(len(k), complex)
        phi_h[hx.hx_indexset_rank(s, spec["target"])] = 1.0
        phi = torch.from_numpy(phi_h).to("cuda")
        args = (s, L, fixed_terms(hx, L), 0)

        def J_of(uu):
            return hx.hx_adjoint_grad(*args, uu, 0.0, spec["T"], spec["substeps"], c0, phi, m=20, gradient=False)[0]

        def central(q, h):
            up, um = u.copy(), u.copy()
            up[q] += h
            um[q] -= h
            return (J_of(up) - J_of(um)) / (2 * h)

        J, g = hx.hx_adjoint_grad(*args, u, 0.0, spec["T"], spec["substeps"], c0, phi, m=20)
        assert 0.0 < J < 1.0
        eps = 1e-13 * J                      # rounding of one evaluation of J
        h = 1e-6
        q = int(np.argmax(np.abs(g)))
        fd = central(q, h)
        assert abs(g[q] - fd) <= 1e-6 * abs(fd) + 2 * eps / h, (q, g[q], fd)
        # smallest entry: Richardson extrapolation, whose rounding error is at most
        # (4 eps / (h/2) + eps / h) / 3 = 3 eps / h for D(h) with step h = 2e-4
        q = int(np.argmin(np.abs(g)))
        rich = (4.0 * central(q, 1e-4) - central(q, 2e-4)) / 3.0
        assert abs(g[q] - rich) <= 1e-6 * abs(g[q]) + 3 * eps / 2e-4, (q, g[q], rich)
    finally:
        hx.hx_indexset_destroy(s)


def test_autograd_function(hx):
    N, B = 3, 40
    L = inputs.half_width(B)
    s = hx.hx_indexset_create(N, B)
    try:
        k = hx.hx_indexset_export(s, N)
        c0 = torch.from_numpy(inputs.coherent_state(k, [0.5, 0.2, 0.0]) / np.linalg.norm(inputs.coherent_state(k, [0.5, 0.2, 0.0]))).to("cuda")
        phi_h = np.zeros(len(k), complex)
        phi_h[hx.hx_indexset_rank(s, [1, 0, 0])] = 1.0
        phi = torch.from_numpy(phi_h).to("cuda")
        f = hx.control_objective(s, L, fixed_terms(hx, L), 0, 0.0, 1.0, 5, c0, phi, m=16)
        u = torch.tensor([0.1, -0.2, 0.05], dtype=torch.float64, requires_grad=True)
        J = f(u)
        J.backward()
        J2, g2 = hx.hx_adjoint_grad(s, L, fixed_terms(hx, L), 0, u.detach().numpy(), 0.0, 1.0, 5, c0, phi, m=16)
        assert abs(J.item() - J2) <= 1e-14
        assert np.allclose(u.grad.numpy(), g2, rtol=0, atol=1e-14)
    finally:
        hx.hx_indexset_destroy(s)


def test_mid_size_gradient_matches_matrix_free_cpu_adjoint(hx, oracle):
    """N = 3, B = 100 (|K| = 1,471), 10 control intervals x 2 sub-steps: the GPU adjoint gradient
    against the oracle's matrix-free FP64 adjoint (Lanczos exponentials and Gauss-Legendre quadrature
    of the Frechet derivative, pinned against scipy's expm_frechet on a tiny set).  Both use m = 32,
    at which the Lanczos exponentials here have converged (a-posteriori estimate about 1e-19)."""
    N, B = 3, 100
    L = inputs.half_width(B)
    S = oracle.IndexSet.hyperbolic(N, B)
    u = np.random.default_rng(6).uniform(-0.1, 0.1, size=10)
    T, substeps = 0.05, 2
    spec = dict(N=N, B=B, L=L, potential=inputs.control_quartic(u, T))
    c0 = inputs.initial_vector({"init": {"kind": "coherent", "q": [1.0, 0.0, 0.0], "eps": 0.0, "seed": 0}}, S.k)
    phi = np.zeros(S.size, complex)
    phi[S.rank([1, 0, 0])] = 1.0
    dt = T / (len(u) * substeps)
    J_ref, g_ref = oracle.control_gradient_matfree(S, spec, c0, phi, dt, len(u) * substeps, len(u), m=32)
    s = hx.hx_indexset_create(N, B)
    try:
        cd = torch.from_numpy(c0).to("cuda")
        pd = torch.from_numpy(phi).to("cuda")
        J, g = hx.hx_adjoint_grad(s, L, fixed_terms(hx, L), 0, u, 0.0, T, substeps, cd, pd, m=32)
    finally:
        hx.hx_indexset_destroy(s)
    assert abs(J - J_ref) <= 1e-12 * abs(J_ref)
    assert np.abs(g - g_ref).max() <= 1e-10 * np.abs(g_ref).max(), np.abs(g - g_ref).max() / np.abs(g_ref).max()
