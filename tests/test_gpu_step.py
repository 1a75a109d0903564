"""GPU parity of the time step (exponential midpoint rule or 2-stage Magnus method, with Lanczos)
against the oracle."""
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


def run_gpu(hx, spec, c0, dtype, dt, nsteps, m=7, t0=0.0, chunks=1, scheme=0):
    P = hx.Problem(spec["N"], spec["B"], dtype=dtype, m=m, scheme=scheme)
    try:
        P.set_potential(spec, t0)
        x = torch.from_numpy(np.ascontiguousarray(c0)).to("cuda", torch.complex128)
        for _ in range(chunks):
            hx.hx_step(P.p, x, dt, nsteps // chunks)
        info = hx.hx_step_info(P.p)
        t = hx.hx_get_time(P.p)
        return x.cpu().numpy(), info, t
    finally:
        P.close()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-12), ("c64", 1e-5)])
def test_henon_heiles_n2_100_steps(hx, oracle, dtype, tol):
    spec = inputs.workload("hh2_b32")
    S = oracle.IndexSet.hyperbolic(2, 32)
    c0 = inputs.initial_vector(spec, S.k)
    ref, t_ref = oracle.expmpr_propagate(S, spec, c0, spec["dt"], spec["steps"], spec["m"])
    dt_ = hx.HX_C128 if dtype == "c128" else hx.HX_C64
    got, info, t = run_gpu(hx, spec, c0, dt_, spec["dt"], spec["steps"], chunks=4)
    assert abs(t - t_ref) < 1e-12
    assert rel(got, ref) <= tol, rel(got, ref)
    assert abs(np.linalg.norm(got) - 1.0) <= (1e-12 if dtype == "c128" else 1e-5)
    assert abs(info["norm"] - np.linalg.norm(got)) < 1e-12


def test_lanczos_coefficients_match_oracle(hx, oracle):
    spec = dict(N=3, B=200, L=inputs.half_width(200), potential=inputs.henon_heiles_chain(3, 0.111, (0.05, 1.0)))
    S = oracle.IndexSet.hyperbolic(3, 200)
    c0 = inputs.initial_vector({"init": {"kind": "coherent", "q": [0.5, -0.3, 0.8], "eps": 1e-3, "seed": 3}}, S.k)
    h = 0.02
    r, a = oracle.potential_terms(spec, 0.5 * h)
    ref, al, be = oracle.lanczos_exp(lambda v: oracle.apply(S, r, a, spec["L"], v), c0, h, 7)
    got, info, _ = run_gpu(hx, spec, c0, hx.HX_C128, h, 1)
    assert info["m_used"] == len(al)
    assert np.allclose(info["alpha"], al, rtol=1e-12, atol=1e-12 * np.abs(al).max())
    assert np.allclose(info["beta"], be, rtol=1e-11)
    assert rel(got, ref) <= 1e-12


def test_harmonic_breakdown_is_exact(hx, oracle):
    """W = 0 and c on three levels of D: Lanczos stops after 3 vectors and the step is exact."""
    spec = dict(N=3, B=30, L=5.0, potential=[])
    S = oracle.IndexSet.hyperbolic(3, 30)
    d = oracle.diag(S)
    c0 = np.zeros(S.size, complex)
    for lev in (1.5, 3.5, 6.5):
        c0[np.where(d == lev)[0]] = 0.3 + 0.1j
    h = 0.37
    got, info, _ = run_gpu(hx, spec, c0, hx.HX_C128, h, 1)
    assert info["breakdown"] and info["m_used"] == 3
    assert np.allclose(got, np.exp(-1j * d * h) * c0, atol=1e-13)


@pytest.mark.parametrize("m", [1, 7, 8])
def test_fused_projections_lanczos_coefficients(hx, oracle, m):
    """complex64 with the specialised product kernel: the kernel computes the first Gram-Schmidt
    projections itself (up to 8 of them, m = 8); T_m and the step still match the oracle to FP32
    accuracy."""
    spec = dict(N=3, B=200, L=inputs.half_width(200), potential=inputs.henon_heiles_chain(3, 0.111, (0.05, 1.0)))
    S = oracle.IndexSet.hyperbolic(3, 200)
    c0 = inputs.initial_vector({"init": {"kind": "coherent", "q": [0.5, -0.3, 0.8], "eps": 1e-3, "seed": 3}}, S.k)
    h = 0.02
    r, a = oracle.potential_terms(spec, 0.5 * h)
    ref, al, be = oracle.lanczos_exp(lambda v: oracle.apply(S, r, a, spec["L"], v), c0, h, m)
    P = hx.Problem(3, 200, dtype=hx.HX_C64, m=m)
    try:
        P.set_potential(spec, 0.0)
        assert hx.hx_apply_specialised(P.p) == 1
        assert hx.hx_step_launches(P.p)[1] == m * 2 + 3       # no separate projection kernel
        x = torch.from_numpy(c0).to("cuda")
        hx.hx_step(P.p, x, h, 1)
        info = hx.hx_step_info(P.p)
        got = x.cpu().numpy()
    finally:
        P.close()
    assert info["m_used"] == len(al) == m
    assert np.allclose(info["alpha"], al, rtol=0, atol=2e-6 * np.abs(al).max())
    assert np.allclose(info["beta"], be, rtol=2e-6)
    assert rel(got, ref) <= 1e-5, rel(got, ref)


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-12), ("c64", 1e-5)])
def test_control_problem_steps(hx, oracle, dtype, tol):
    spec = inputs.workload("ctrl4_b512")
    S = oracle.IndexSet.hyperbolic(4, 512)
    c0 = inputs.initial_vector(spec, S.k)
    h = 0.005
    ref, _ = oracle.expmpr_propagate(S, spec, c0, h, 20, 7, t0=0.03)
    got, _, _ = run_gpu(hx, spec, c0, hx.HX_C128 if dtype == "c128" else hx.HX_C64, h, 20, t0=0.03)
    assert rel(got, ref) <= tol, rel(got, ref)


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-12), ("c64", 1e-5)])
def test_full_size_one_step(hx, oracle, dtype, tol):
    """One step of the N=6, B=4096 workload (|K| = 4,883,360) against the oracle."""
    spec = inputs.workload("hh6_b4096")
    S = oracle.IndexSet.hyperbolic(6, 4096)
    c0 = inputs.initial_vector(spec, S.k)
    ref, _ = oracle.expmpr_propagate(S, spec, c0, spec["dt"], 1, spec["m"])
    got, _, _ = run_gpu(hx, spec, c0, hx.HX_C128 if dtype == "c128" else hx.HX_C64, spec["dt"], 1)
    assert rel(got, ref) <= tol, rel(got, ref)


def test_backward_step_returns_to_the_start(hx, oracle):
    """A step with -dt from t + dt evaluates A at the same midpoint: it undoes the step up to the
    Lanczos error (here far below 1e-12), and each matches the oracle's step with its sign of dt."""
    spec = inputs.workload("hh2_b32")
    S = oracle.IndexSet.hyperbolic(2, 32)
    c0 = inputs.initial_vector(spec, S.k)
    fwd, _ = oracle.expmpr_propagate(S, spec, c0, 0.01, 1, 7)
    P = hx.Problem(2, 32)
    try:
        P.set_potential(spec, 0.0)
        x = torch.from_numpy(c0.copy()).to("cuda")
        hx.hx_step(P.p, x, 0.01, 1)
        assert rel(x.cpu().numpy(), fwd) <= 1e-12
        hx.hx_step(P.p, x, -0.01, 1)
        assert abs(hx.hx_get_time(P.p)) < 1e-15
        back = x.cpu().numpy()
    finally:
        P.close()
    ref_back, _ = oracle.expmpr_propagate(S, spec, fwd, -0.01, 1, 7, t0=0.01)
    assert rel(back, ref_back) <= 1e-12
    assert rel(back, c0) <= 1e-10


def test_host_step_on_pinned_memory(hx, oracle):
    """hx_step_host on page-locked memory (the bench's end-to-end path), one and two steps, against
    the oracle."""
    spec = inputs.workload("hh2_b32")
    S = oracle.IndexSet.hyperbolic(2, 32)
    c0 = inputs.initial_vector(spec, S.k)
    ref1, _ = oracle.expmpr_propagate(S, spec, c0, 0.01, 1, 7)
    ref3, _ = oracle.expmpr_propagate(S, spec, c0, 0.01, 3, 7)
    P = hx.Problem(2, 32)
    try:
        P.set_potential(spec, 0.0)
        pinned = torch.from_numpy(c0.copy()).pin_memory()
        c = pinned.numpy()
        hx.hx_step_host(P.p, c, 0.01, 1)
        assert rel(c, ref1) <= 1e-12
        hx.hx_step_host(P.p, c, 0.01, 2)
        assert rel(c, ref3) <= 1e-12
        assert abs(hx.hx_get_time(P.p) - 0.03) < 1e-14
    finally:
        P.close()


def test_host_step_entry_point(hx, oracle):
    spec = inputs.workload("hh2_b32")
    S = oracle.IndexSet.hyperbolic(2, 32)
    c0 = inputs.initial_vector(spec, S.k)
    ref, _ = oracle.expmpr_propagate(S, spec, c0, 0.01, 5, 7)
    P = hx.Problem(2, 32)
    try:
        P.set_potential(spec, 0.0)
        c = c0.copy()
        hx.hx_step_host(P.p, c, 0.01, 5)
        assert rel(c, ref) <= 1e-12
    finally:
        P.close()


def _laser_hh(N, B):
    """Henon-Heiles chain with a strong sin^2(2t) x_1 term: A(t) varies on the time scale of a step."""
    return dict(N=N, B=B, L=inputs.half_width(B),
                potential=inputs.henon_heiles_chain(N, 0.2) + [{"coef": 0.8, "powers": {0: 1},
                                                                "mod": {"kind": "sin2", "omega": 2.0}}])


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-12), ("c64", 1e-5)])
@pytest.mark.parametrize("N,B,h,steps", [(2, 40, 0.05, 20), (4, 60, 0.02, 10)])
def test_magnus4_matches_oracle(hx, oracle, dtype, tol, N, B, h, steps):
    """Eq. (2stageMagnus): four products per Lanczos vector at the two Gauss-Legendre times.  The
    cases keep h |H| small enough for m = 7 to converge: there the step map does not amplify
    rounding (a 1e-10 perturbation of c0 grows by at most 1.02 over the run; at N = 4, B = 300,
    h = 0.05 it grows by 1.5e5, and two correct implementations differ by that factor times their
    rounding)."""
    spec = _laser_hh(N, B)
    S = oracle.IndexSet.hyperbolic(N, B)
    c0 = inputs.initial_vector({"init": {"kind": "coherent", "q": [0.6] * N, "eps": 1e-3, "seed": 5}}, S.k)
    ref, t_ref = oracle.magnus4_propagate(S, spec, c0, h, steps, 7, t0=0.1)
    dt_ = hx.HX_C128 if dtype == "c128" else hx.HX_C64
    got, info, t = run_gpu(hx, spec, c0, dt_, h, steps, t0=0.1, chunks=2, scheme=hx.HX_SCHEME_MAGNUS4)
    assert abs(t - t_ref) < 1e-12
    assert rel(got, ref) <= tol, rel(got, ref)
    if dtype == "c128":                       # the two schemes differ by far more than the tolerance
        mpr, _ = oracle.expmpr_propagate(S, spec, c0, h, steps, 7, t0=0.1)
        assert rel(mpr, ref) > 1e3 * tol


def _drifting(N, B):
    """beta cos(x_d - x_{d+1} + omega t) chain: the interpolant's shape changes with t."""
    return dict(N=N, B=B, L=inputs.half_width(B), potential=inputs.drifting_cos_chain(N, 0.2, 2.0))


@pytest.mark.parametrize("h", [0.02, -0.02])
@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("dtype,tol", [("c128", 1e-12), ("c64", 1e-5)])
def test_reinterpolated_potential_matches_oracle(hx, oracle, scheme, dtype, tol, h):
    """The time-propagation algorithm of Sec. 2.2 with its step (1) every step: the potential's
    degree-8 Chebyshev interpolant is computed anew at t + h/2 (exponential midpoint rule) or at the
    two Gauss-Legendre points (2-stage Magnus method) through hx_step_reinterp; the oracle
    interpolates at the same times.  Also backwards in time (h < 0)."""
    N, B, steps, t0 = 3, 60, 10, 0.1
    spec = _drifting(N, B)
    S = oracle.IndexSet.hyperbolic(N, B)
    c0 = inputs.initial_vector({"init": {"kind": "coherent", "q": [0.5, -0.3, 0.2], "eps": 1e-3, "seed": 6}}, S.k)
    prop = oracle.magnus4_propagate if scheme else oracle.expmpr_propagate
    ref, t_ref = prop(S, spec, c0, h, steps, 7, t0=t0)
    P = hx.Problem(N, B, dtype=hx.HX_C128 if dtype == "c128" else hx.HX_C64, scheme=scheme)
    try:
        x = torch.from_numpy(np.ascontiguousarray(c0)).to("cuda", torch.complex128)
        hx.hx_set_time(P.p, t0)
        P.step_reinterp(spec, x, h, steps)
        t = hx.hx_get_time(P.p)
        got = x.cpu().numpy()
    finally:
        P.close()
    assert abs(t - t_ref) < 1e-12
    assert rel(got, ref) <= tol, rel(got, ref)
    if dtype == "c128":          # the change of shape matters far beyond the tolerance
        frozen = dict(spec, potential=[dict(c, omega=0.0) for c in spec["potential"]])
        assert rel(prop(S, frozen, c0, h, steps, 7, t0=t0)[0], ref) > 1e3 * tol


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_reinterpolating_a_fixed_potential_is_hx_step(hx, dtype):
    """With a potential that does not change, the per-step path runs the kernels hx_step runs on
    the same arguments: the states agree bit for bit."""
    spec = inputs.workload("hh2_b32")
    dt_ = hx.HX_C128 if dtype == "c128" else hx.HX_C64
    P, Q = hx.Problem(2, 32, dtype=dt_), hx.Problem(2, 32, dtype=dt_)
    try:
        P.set_potential(spec, 0.0)
        c0 = inputs.initial_vector(spec, hx.hx_indexset_export(P.set, 2))
        a = torch.from_numpy(c0).to("cuda")
        b = a.clone()
        hx.hx_step(P.p, a, 0.01, 5)
        Q.step_reinterp(spec, b, 0.01, 5)
        torch.cuda.synchronize()
        assert torch.equal(a, b)
        assert hx.hx_get_time(Q.p) == pytest.approx(0.05, abs=1e-14)
    finally:
        P.close()
        Q.close()


def test_reinterp_argument_errors(hx):
    import ctypes
    P = hx.Problem(2, 40, scheme=hx.HX_SCHEME_MAGNUS4)
    try:
        x = torch.zeros(P.size, dtype=torch.complex128, device="cuda")
        nothing = hx.POTENTIAL_FN(lambda t, u: None)
        assert hx.lib.hx_step_reinterp(P.p, ctypes.c_void_p(x.data_ptr()), 0.01, 1, nothing, None) == hx.HX_EINVAL
        assert "no potential" in hx.hx_last_error()
        with pytest.raises(hx.HxError):      # Magnus needs constant terms (it switches them per Gauss point)
            P.step_reinterp(_laser_hh(2, 40), x, 0.01, 1)
        assert hx.lib.hx_step_reinterp(P.p, ctypes.c_void_p(x.data_ptr() + 8), 0.01, 1, nothing, None) == hx.HX_EINVAL
    finally:
        P.close()


def test_magnus4_time_integration_experiment(hx, oracle):
    """The time-integration experiment of Sec. 6.3 (N = 2, K = 40, m = 7, h = 1/10) on the GPU equals
    the oracle's 2-stage Magnus run (whose error against the exact-Galerkin solution the oracle pins
    reproduce from the paper's table)."""
    spec = inputs.time_integration_workload(2, 40)
    S = oracle.IndexSet.hyperbolic(2, spec["B"])
    c0 = inputs.initial_vector(spec, S.k)
    ref, _ = oracle.magnus4_propagate(S, spec, c0, 0.1, 10, 7)
    got, _, t = run_gpu(hx, spec, c0, hx.HX_C128, 0.1, 10, scheme=hx.HX_SCHEME_MAGNUS4)
    assert abs(t - 1.0) < 1e-12
    assert rel(got, ref) <= 1e-12, rel(got, ref)


def test_step_launch_counts(hx):
    # expMPR: the specialised complex64 product kernel computes the projections itself when m <= 8
    # and the product is one launch; Magnus: the two-time kernels need a one-stage product too
    # Gram-Schmidt: one sweep per vector for m <= 8 (then start, exponential, recombination: 3),
    # two passes for m > 8 (the last vector's second pass skipped: 2)
    def gs(m):
        return 1 if m <= 8 else 2

    def fixed(m):
        return 3 if m <= 8 else 2

    per = {0: lambda m, a, spec, c64: m * (a + gs(m) + (0 if spec and c64 and m <= 8 and a == 1 else 1)) + fixed(m),
           1: lambda m, a, spec, c64: m * ((2 * a if spec and a == 1 else 4 * a + 1) + 1 + gs(m)) + fixed(m)}
    for scheme in (0, 1):
        for name in ("hh2_b32", "cos10_b1024"):
            spec = inputs.workload(name) if name == "hh2_b32" else dict(N=3, B=40, L=inputs.half_width(40),
                                                                      potential=inputs.cos_chain(3, 0.2, 8))
            for m, dtype in ((6, hx.HX_C64), (6, hx.HX_C128), (12, hx.HX_C64)):
                P = hx.Problem(spec["N"], spec["B"], m=m, scheme=scheme, dtype=dtype)
                try:
                    P.set_potential(spec, 0.0)
                    a, step = hx.hx_step_launches(P.p)
                    assert a == (1 if name == "hh2_b32" else 2)
                    specialised = hx.hx_apply_specialised(P.p)
                    assert specialised == 1        # the cosine chain's channel stage is compiled too
                    assert step == per[scheme](m, a, specialised, dtype == hx.HX_C64)
                finally:
                    P.close()


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-12), ("c64", 2e-6)])
def test_energy_matches_oracle_and_is_conserved(hx, oracle, dtype, tol):
    """hx_energy = <c, A c> against the oracle's product; for a time-independent W the exponential
    midpoint rule keeps the energy (and the norm) up to the Lanczos error over 50 steps."""
    spec = inputs.workload("hh2_b32")
    S = oracle.IndexSet.hyperbolic(2, 32)
    c0 = inputs.initial_vector(spec, S.k)
    r, a = oracle.potential_terms(spec, 0.0)
    e_ref = float(np.real(np.vdot(c0, oracle.apply(S, r, a, spec["L"], c0))))
    P = hx.Problem(2, 32, dtype=hx.HX_C128 if dtype == "c128" else hx.HX_C64)
    try:
        P.set_potential(spec, 0.0)
        x = torch.from_numpy(c0.copy()).to("cuda", torch.complex128 if dtype == "c128" else torch.complex64)
        e0 = hx.hx_energy(P.p, x)
        assert abs(e0 - e_ref) <= tol * abs(e_ref), (e0, e_ref)
        if dtype == "c128":
            hx.hx_step(P.p, x, 0.01, 50)
            assert abs(hx.hx_energy(P.p, x) - e0) <= 1e-10 * abs(e0)
    finally:
        P.close()


def test_fig8_perturbed_lanczos_row_on_gpu(hx, oracle):
    """Sec. 6.2, Fig. 8, row N = 4, K = 40 (m = 5, h = 1/10 and 1/20): the GPU step (fast product,
    complex128) against the Lanczos step with the exact Galerkin matrix of the interpolated torsional
    potential reproduces the printed perturbation errors (read with max-abs, as Fig. 5); the GPU step
    itself matches the oracle's fast-product step to 1e-12."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "fig8_perturbed_lanczos.json")))
    row = next(r for r in gold["rows"] if r["N"] == 4 and r["K"] == 40)
    N, K = 4, 40
    comps = [{"coef": -1.0, "func": "cos_scaled", "axes": [l], "scale": 1 / 16.0, "R": 8} for l in range(N)]
    spec = dict(N=N, B=K + 1, L=16.0, potential=comps + [{"coef": float(N), "powers": {}}])
    S = oracle.IndexSet.hyperbolic(N, K + 1)
    r, a = oracle.potential_terms(spec, 0.0)
    v = inputs.initial_vector({"init": {"kind": "beta_decay", "beta": gold["beta"]}}, S.k)
    d = oracle.diag(S)
    A = np.diag(d) + oracle.gh_assembly(S, r, a, 16.0, K + 10)
    for h, printed in zip(gold["h"][:2], row["err"][:2]):
        up, _, _ = oracle.lanczos_exp(lambda x: A @ x, v, h, gold["m"])
        pe, _, _ = oracle.lanczos_exp(lambda x: oracle.apply(S, r, a, 16.0, x), v, h, gold["m"])
        got, _, _ = run_gpu(hx, spec, v, hx.HX_C128, h, 1, m=gold["m"])
        assert rel(got, pe) <= 1e-12, rel(got, pe)
        err = np.abs(up - got).max()
        assert err == pytest.approx(printed, rel=5e-3), (h, err, printed)


@pytest.mark.parametrize("m,h", [(8, 10.0), (5, 12.0), (3, 20.0)])
def test_large_step_exponential_matches_oracle(hx, oracle, m, h):
    """|h| ||T_m|| beyond the Chebyshev series' range (> 96): the exponential takes the eigenpair path
    (FP32 bisection, FP64 Newton and inverse iteration, or the QL fallback); one step against the
    oracle's eigendecomposition of T_m."""
    spec = inputs.workload("hh2_b32")
    S = oracle.IndexSet.hyperbolic(2, 32)
    c0 = inputs.initial_vector(spec, S.k)
    ref, _ = oracle.expmpr_propagate(S, spec, c0, h, 1, m)
    got, info, _ = run_gpu(hx, spec, c0, hx.HX_C128, h, 1, m=m)
    assert info["m_used"] == m
    assert h * (max(info["alpha"]) - min(info["alpha"])) / 2 > 96
    assert rel(got, ref) <= 1e-12, rel(got, ref)


@pytest.mark.parametrize("N,B", [(1, 1), (3, 1), (1, 50), (2, 3)])
@pytest.mark.parametrize("dtype,tol", [("c128", 1e-12), ("c64", 1e-5)])
def test_tiny_problems_step(hx, oracle, N, B, dtype, tol):
    """Index sets of 1 to 50 elements (fewer than a warp or a pair, odd lengths): the product with its
    projections, the Gram-Schmidt passes, the exponential and the recombination at their smallest
    sizes, with the Lanczos process stopping early when the Krylov space is exhausted."""
    comps = [{"coef": 0.3, "powers": {0: 3}}, {"coef": -0.2, "powers": {0: 1}}]
    if N > 1:
        comps.append({"coef": 0.1, "powers": {0: 2, N - 1: 1}})
    spec = dict(N=N, B=B, L=inputs.half_width(max(B, 2)), potential=comps)
    S = oracle.IndexSet.hyperbolic(N, B)
    c0 = inputs.initial_vector({"init": {"kind": "gaussian", "seed": 9}}, S.k)
    ref, _ = oracle.expmpr_propagate(S, spec, c0, 0.05, 3, 7)
    got, info, _ = run_gpu(hx, spec, c0, hx.HX_C128 if dtype == "c128" else hx.HX_C64, 0.05, 3)
    assert info["m_used"] == min(7, S.size) or info["breakdown"]
    assert rel(got, ref) <= tol, rel(got, ref)


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-12), ("c64", 1e-5)])
def test_cosine_chain_n10_steps(hx, oracle, dtype, tol):
    """The N = 10 cosine chain (degree-8 Chebyshev interpolant of 0.2 sum cos(x_d - x_{d+1})) at a
    reduced bound B = 32 (9,533 coefficients, so that the oracle's term-by-term evaluation of the
    9 x 9 tensor interpolants stays within seconds): its degree-8 plane terms take the two-stage path
    through channel vectors (footprint above the direct limit), three steps against the oracle."""
    base = inputs.workload("cos10_b1024")
    spec = dict(base, B=32, L=inputs.half_width(32))
    S = oracle.IndexSet.hyperbolic(10, 32)
    c0 = inputs.initial_vector(spec, S.k)
    ref, t_ref = oracle.expmpr_propagate(S, spec, c0, spec["dt"], 3, spec["m"])
    dt_ = hx.HX_C128 if dtype == "c128" else hx.HX_C64
    P = hx.Problem(10, 32, dtype=dt_, m=spec["m"])
    try:
        P.set_potential(spec, 0.0)
        assert hx.hx_step_launches(P.p)[0] == 2          # channel stage + main stage
        x = torch.from_numpy(np.ascontiguousarray(c0)).to("cuda", torch.complex128)
        hx.hx_step(P.p, x, spec["dt"], 3)
        got = x.cpu().numpy()
    finally:
        P.close()
    assert rel(got, ref) <= tol, rel(got, ref)
