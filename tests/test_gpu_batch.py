"""GPU batches of independent problems (hx_batch_*): same result as stepping each problem alone, and
parity with the oracle on sampled members."""
import contextlib
import os

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


@contextlib.contextmanager
def generic_kernel():
    """Problems whose potential is set inside run the generic product kernel, the one batch steps
    run: bit-identical results need the same kernels (the specialised complex64 kernel also fuses
    the Lanczos projections, which sums them in another order)."""
    old = os.environ.get("HX_APPLY_SPECIALISE")
    os.environ["HX_APPLY_SPECIALISE"] = "0"
    try:
        yield
    finally:
        if old is None:
            del os.environ["HX_APPLY_SPECIALISE"]
        else:
            os.environ["HX_APPLY_SPECIALISE"] = old


def test_batch_equals_individual_steps_and_oracle(hx, oracle):
    specs = inputs.batch_workloads(n=16, seed=3, b_lo=64, b_hi=600)
    dtypes = [hx.HX_C64 if i % 4 else hx.HX_C128 for i in range(len(specs))]
    probs, alone, states, states_alone, c0s = [], [], [], [], []
    try:
        for spec, dt_ in zip(specs, dtypes):
            P = hx.Problem(spec["N"], spec["B"], dtype=dt_, m=spec["m"])
            P.set_potential(spec, 0.0)
            Q = hx.Problem(spec["N"], spec["B"], dtype=dt_, m=spec["m"], indexset=P.set)
            with generic_kernel():
                Q.set_potential(spec, 0.0)
            k = hx.hx_indexset_export(P.set, spec["N"])
            c0 = inputs.initial_vector(spec, k)
            c0s.append(c0)
            probs.append(P)
            alone.append(Q)
            states.append(torch.from_numpy(c0).to("cuda"))
            states_alone.append(torch.from_numpy(c0).to("cuda"))
        b = hx.hx_batch_create([P.p for P in probs])
        try:
            hx.hx_batch_step(b, states, 0.01, 7)
            hx.hx_batch_step(b, states, 0.01, 13)      # replays the same graph
        finally:
            hx.hx_batch_destroy(b)
        for Q, c in zip(alone, states_alone):
            hx.hx_step(Q.p, c, 0.01, 20)
        torch.cuda.synchronize()
        for P, Q, c, ca in zip(probs, alone, states, states_alone):
            assert torch.equal(c, ca)
            assert abs(hx.hx_get_time(P.p) - 0.2) < 1e-12
        for i in (0, 5, 11):           # a complex128 member and two complex64 members
            spec = specs[i]
            S = oracle.IndexSet.hyperbolic(spec["N"], spec["B"])
            ref, _ = oracle.expmpr_propagate(S, spec, c0s[i], 0.01, 20, spec["m"])
            got = states[i].cpu().numpy()
            tol = 1e-12 if dtypes[i] == hx.HX_C128 else 1e-5
            assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= tol, i
    finally:
        for P in alone + probs:
            P.close()


def test_batch_argument_errors(hx):
    spec = inputs.workload("hh2_b32")
    P = hx.Problem(2, 32)
    try:
        with pytest.raises(hx.HxError):
            hx.hx_batch_create([P.p])               # no potential yet
        P.set_potential(spec, 0.0)
        with pytest.raises(hx.HxError):
            hx.hx_batch_create([P.p, P.p])          # the same problem twice
        Q = hx.Problem(2, 32)
        try:
            Q.set_potential(spec, 0.0)
            b = hx.hx_batch_create([P.p, Q.p])
            try:
                buf = torch.zeros(2 * P.size, dtype=torch.complex128, device="cuda")
                with pytest.raises(hx.HxError):     # one state for both members
                    hx.hx_batch_step(b, [buf[: P.size], buf[: P.size]], 0.01, 1)
                with pytest.raises(hx.HxError):     # states sharing one element
                    hx.hx_batch_step(b, [buf[1: P.size + 1], buf[: P.size]], 0.01, 1)
                hx.hx_batch_step(b, [buf[: P.size], buf[P.size:]], 0.01, 0)
            finally:
                hx.hx_batch_destroy(b)
        finally:
            Q.close()
    finally:
        P.close()


def test_batch_follows_potential_change(hx):
    """Setting a member's potential again after a batch step makes the next batch step use it."""
    spec = inputs.workload("hh2_b32")
    spec2 = dict(spec, potential=inputs.henon_heiles_chain(2, 0.05, None))
    P, Q = hx.Problem(2, 32), hx.Problem(2, 32)
    try:
        P.set_potential(spec, 0.0)
        k = hx.hx_indexset_export(P.set, 2)
        c0 = inputs.initial_vector(spec, k)
        c, ca = torch.from_numpy(c0).to("cuda"), torch.from_numpy(c0).to("cuda")
        b = hx.hx_batch_create([P.p])
        try:
            hx.hx_batch_step(b, [c], 0.01, 3)
            P.set_potential(spec2, hx.hx_get_time(P.p))
            hx.hx_batch_step(b, [c], 0.01, 3)
        finally:
            hx.hx_batch_destroy(b)
        with generic_kernel():
            Q.set_potential(spec, 0.0)
        hx.hx_step(Q.p, ca, 0.01, 3)
        with generic_kernel():
            Q.set_potential(spec2, hx.hx_get_time(Q.p))
        hx.hx_step(Q.p, ca, 0.01, 3)
        torch.cuda.synchronize()
        assert torch.equal(c, ca)
    finally:
        P.close()
        Q.close()
