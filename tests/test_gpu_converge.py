"""Converged time steps: the a-posteriori error estimate of the Lanczos exponential (Sec. 2.2),
automatic sub-steps (hx_config.tol), converged runs against the oracle and mixed precision
against FP64 over the Henon-Heiles chain's 1000 steps, and the reporting of non-finite values."""
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


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def oracle_substeps(oracle, S, spec, c, t, dt, s, m):
    """One step of size dt as s sub-steps of the exponential midpoint rule; the largest estimate."""
    h = dt / s
    est = 0.0
    for j in range(s):
        r, a = oracle.potential_terms(spec, t + (j + 0.5) * h)
        c, _, _, e = oracle.lanczos_exp(lambda v: oracle.apply(S, r, a, spec["L"], v), c, h, m, estimate=True)
        est = max(est, e)
    return c, est


@pytest.mark.parametrize("dtype,tol_state", [("c128", 1e-12), ("c64", 1e-5)])
def test_adaptive_substeps_match_oracle(hx, oracle, dtype, tol_state):
    """N = 2 Henon-Heiles with dt = 0.1 (h ||A|| about 4 per step, m = 7 unresolved): each step is
    split until the estimate is at most 1e-10; the oracle takes the same sub-steps and gives the
    same states and the same estimates."""
    spec = inputs.workload("hh2_b32")
    S = oracle.IndexSet.hyperbolic(2, 32)
    c0 = inputs.initial_vector(spec, S.k)
    dt, nsteps, m, tol = 0.1, 6, 7, 1e-10
    P = hx.Problem(2, 32, dtype=hx.HX_C128 if dtype == "c128" else hx.HX_C64, m=m, tol=tol)
    try:
        P.set_potential(spec, 0.0)
        x = torch.from_numpy(c0.copy()).to("cuda")
        c, t, subs = c0.copy(), 0.0, []
        for _ in range(nsteps):
            hx.hx_step(P.p, x, dt, 1)
            st = hx.hx_step_substeps(P.p)
            subs.append(st["last"])
            assert st["total"] == st["last"]
            c, est = oracle_substeps(oracle, S, spec, c, t, dt, st["last"], m)
            t += dt
            assert st["err_max"] <= tol
            assert est <= tol
            if dtype == "c128":
                assert abs(st["err_max"] - est) <= 1e-6 * est + 1e-300, (st["err_max"], est)
        assert max(subs) > 1, subs                 # the tolerance forced sub-steps
        assert abs(hx.hx_get_time(P.p) - t) < 1e-12
        assert rel(x.cpu().numpy(), c) <= tol_state, rel(x.cpu().numpy(), c)
    finally:
        P.close()


def test_substeps_without_tolerance(hx):
    """tol = 0: one Lanczos exponential per step, reported as one sub-step per step."""
    spec = inputs.workload("hh2_b32")
    P = hx.Problem(2, 32, dtype=hx.HX_C128)
    try:
        P.set_potential(spec, 0.0)
        x = torch.zeros(P.size, dtype=torch.complex128, device="cuda")
        x[0] = 1.0
        hx.hx_step(P.p, x, 0.01, 5)
        assert hx.hx_step_substeps(P.p) == {"last": 1, "total": 5, "err_max": 0.0}
    finally:
        P.close()


def test_looser_tolerance_takes_fewer_substeps(hx):
    spec = inputs.workload("hh2_b32")
    totals = []
    for tol in (1e-12, 1e-6):
        P = hx.Problem(2, 32, dtype=hx.HX_C128, tol=tol)
        try:
            P.set_potential(spec, 0.0)
            x = torch.zeros(P.size, dtype=torch.complex128, device="cuda")
            x[3] = 1.0
            hx.hx_step(P.p, x, 0.2, 4)
            totals.append(hx.hx_step_substeps(P.p)["total"])
        finally:
            P.close()
    assert totals[0] > totals[1] >= 4, totals


def test_converged_full_size_steps_match_oracle(hx, oracle):
    """The Henon-Heiles chain at N = 6, B = 4096 (4,883,360 coefficients) with dt = 2.5e-5: three
    steps whose Lanczos exponentials meet the estimate 1e-6, FP64, against the oracle taking the
    same sub-steps (the step map is then close to unitary, so rounding does not grow)."""
    spec = inputs.workload("hh6_b4096")
    S = oracle.IndexSet.hyperbolic(spec["N"], spec["B"])
    c0 = inputs.initial_vector(spec, S.k)
    dt, m, tol = spec["dt_converged"], 7, 1e-6
    P = hx.Problem(spec["N"], spec["B"], dtype=hx.HX_C128, m=m, tol=tol)
    try:
        P.set_potential(spec, 0.0)
        x = torch.from_numpy(c0.copy()).to("cuda")
        c, t = c0.copy(), 0.0
        for _ in range(3):
            hx.hx_step(P.p, x, dt, 1)
            s = hx.hx_step_substeps(P.p)["last"]
            assert s <= 2, s                      # the oracle's time stays bounded
            c, est = oracle_substeps(oracle, S, spec, c, t, dt, s, m)
            t += dt
            assert est <= tol
        assert rel(x.cpu().numpy(), c) <= 1e-12, rel(x.cpu().numpy(), c)
    finally:
        P.close()


def test_mixed_vs_fp64_henon_heiles_1000_steps(hx, oracle):
    """The chain's 1000 steps (dt = 2.5e-5, every Lanczos exponential within the estimate 1e-6): the
    complex64 stencil with FP64 reductions stays within 1e-5 of the FP64 run."""
    spec = inputs.workload("hh6_b4096")
    c0 = inputs.initial_vector(spec, oracle.IndexSet.hyperbolic(spec["N"], spec["B"]).k)
    out = {}
    for name, dt_ in (("c128", hx.HX_C128), ("c64", hx.HX_C64)):
        P = hx.Problem(spec["N"], spec["B"], dtype=dt_, m=7, tol=1e-6)
        try:
            P.set_potential(spec, 0.0)
            x = torch.from_numpy(c0.copy()).to("cuda")
            hx.hx_step(P.p, x, spec["dt_converged"], spec["steps"])
            out[name] = x.cpu().numpy()
            assert hx.hx_step_substeps(P.p)["err_max"] <= 1e-6
        finally:
            P.close()
    assert rel(out["c64"], out["c128"]) <= 1e-5, rel(out["c64"], out["c128"])
    assert abs(np.linalg.norm(out["c128"]) - np.linalg.norm(c0)) <= 1e-10 * np.linalg.norm(c0)


def test_nan_in_state_is_reported(hx):
    """A NaN planted on the host in the state: the step reports HX_ENONFINITE, and so does hx_norm."""
    spec = inputs.workload("hh2_b32")
    for dtype in (hx.HX_C128, hx.HX_C64):
        P = hx.Problem(2, 32, dtype=dtype)
        try:
            P.set_potential(spec, 0.0)
            c = np.ones(P.size, dtype=np.complex128) / np.sqrt(P.size)
            c[5] = np.nan
            x = torch.from_numpy(c).to("cuda")
            v = x.to(torch.complex64) if dtype == hx.HX_C64 else x.clone()
            with pytest.raises(hx.HxError) as ei:
                hx.hx_norm(P.p, v)
            assert ei.value.status == hx.HX_ENONFINITE
            hx.hx_step(P.p, x, 0.01, 2)
            with pytest.raises(hx.HxError) as ei:
                hx.hx_step_info(P.p)
            assert ei.value.status == hx.HX_ENONFINITE
        finally:
            P.close()


def test_nan_in_potential_coefficient_is_reported(hx):
    """A NaN planted in one coefficient alpha of the potential: the step reports HX_ENONFINITE."""
    spec = dict(inputs.workload("hh2_b32"))
    spec["potential"] = list(spec["potential"]) + [{"coef": float("nan"), "powers": {1: 2}}]
    P = hx.Problem(2, 32, dtype=hx.HX_C128)
    try:
        P.set_potential(spec, 0.0)
        x = torch.zeros(P.size, dtype=torch.complex128, device="cuda")
        x[0] = 1.0
        hx.hx_step(P.p, x, 0.01, 1)
        with pytest.raises(hx.HxError) as ei:
            hx.hx_step_info(P.p)
        assert ei.value.status == hx.HX_ENONFINITE
    finally:
        P.close()


def test_wrong_vector_type_or_length_refused(hx):
    """The binding refuses, on the host, a vector of another type than the problem's or shorter
    than |K| (the library would read past its end)."""
    spec = inputs.workload("hh2_b32")
    P = hx.Problem(2, 32, dtype=hx.HX_C128)
    try:
        P.set_potential(spec, 0.0)
        ok = torch.zeros(P.size, dtype=torch.complex128, device="cuda")
        with pytest.raises(ValueError):
            hx.hx_apply(P.p, torch.zeros(P.size, dtype=torch.complex64, device="cuda"), ok)
        with pytest.raises(ValueError):
            hx.hx_norm(P.p, torch.zeros(P.size - 1, dtype=torch.complex128, device="cuda"))
        with pytest.raises(ValueError):
            hx.hx_step(P.p, torch.zeros(P.size, dtype=torch.complex64, device="cuda"), 0.01, 1)
    finally:
        P.close()


def test_mixed_vs_fp64_cosine_chain_500_steps(hx):
    """The N = 10, B = 1024 cosine chain (8,996,478 coefficients, degree-8 interpolants through channel
    vectors) over its 500 steps at the converged step 1e-3 (every Lanczos exponential within the
    estimate 1e-6): the complex64 stencil with FP64 reductions stays within 1e-5 of the FP64 run."""
    spec = inputs.workload("cos10_b1024")
    s = hx.hx_indexset_create(spec["N"], spec["B"])
    try:
        c0 = inputs.initial_vector(spec, hx.hx_indexset_export(s, spec["N"]))
        out = {}
        for name, dt_ in (("c128", hx.HX_C128), ("c64", hx.HX_C64)):
            P = hx.Problem(spec["N"], spec["B"], dtype=dt_, m=7, tol=1e-6, indexset=s)
            try:
                P.set_potential(spec, 0.0)
                x = torch.from_numpy(c0.copy()).to("cuda")
                hx.hx_step(P.p, x, spec["dt_converged"], spec["steps"])
                out[name] = x.cpu().numpy()
                assert hx.hx_step_substeps(P.p)["err_max"] <= 1e-6
            finally:
                P.close()
    finally:
        hx.hx_indexset_destroy(s)
    assert rel(out["c64"], out["c128"]) <= 1e-5, rel(out["c64"], out["c128"])
