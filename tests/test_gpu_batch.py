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


@contextlib.contextmanager
def env(name, value):
    old = os.environ.get(name)
    if value is None:
        os.environ.pop(name, None)
    else:
        os.environ[name] = value
    try:
        yield
    finally:
        if old is None:
            os.environ.pop(name, None)
        else:
            os.environ[name] = old


def mixed_batch_specs():
    """Twelve small members: both precisions, Krylov dimensions 5 and 7, and two members with a
    degree-4 term (the degree-8 class of the batched product kernel)."""
    specs = inputs.batch_workloads(n=12, seed=11, b_lo=48, b_hi=900)
    for i, s in enumerate(specs):
        if i % 3 == 1:
            s["m"] = 5
        if i in (2, 7):
            s["potential"] = s["potential"] + [{"coef": 0.004, "powers": {0: 4}}]
    return specs


def run_batch(hx, specs, dtypes, nsteps=(4, 5), budget=None, batched="1", infos=None):
    probs, states, c0s = [], [], []
    try:
        for spec, dt_ in zip(specs, dtypes):
            P = hx.Problem(spec["N"], spec["B"], dtype=dt_, m=spec["m"])
            P.set_potential(spec, 0.0)
            c0 = inputs.initial_vector(spec, hx.hx_indexset_export(P.set, spec["N"]))
            probs.append(P)
            c0s.append(c0)
            states.append(torch.from_numpy(c0).to("cuda"))
        b = hx.hx_batch_create([P.p for P in probs])
        try:
            if budget is not None:
                hx.hx_batch_set_budget(b, budget)
            with env("HX_BATCH_BATCHED", batched):
                for n in nsteps:
                    hx.hx_batch_step(b, states, 0.01, n)
                    if infos is not None:
                        infos.append(hx.hx_batch_info(b))
            info = hx.hx_batch_info(b)
        finally:
            hx.hx_batch_destroy(b)
        torch.cuda.synchronize()
        return [s.cpu().numpy() for s in states], c0s, info
    finally:
        for P in probs:
            P.close()


def test_batched_products_equal_member_graphs_and_oracle(hx, oracle):
    """The batched product launches (one per Lanczos index and class, tiles of all members) give the
    same bits as one graph per member with its own product launches, for members of both precisions,
    two Krylov dimensions and both degree classes; one member of each precision against the oracle."""
    specs = mixed_batch_specs()
    dtypes = [hx.HX_C64 if i % 4 else hx.HX_C128 for i in range(len(specs))]
    got, c0s, info = run_batch(hx, specs, dtypes, batched="1")
    ref, _, info0 = run_batch(hx, specs, dtypes, batched="0")
    assert info["batched"] and not info0["batched"]
    assert info["schedule"] == hx.HX_SCHED_BATCHED and info0["schedule"] == hx.HX_SCHED_MEMBERS
    assert info["launches"] > 0 and info0["launches"] > info["launches"]
    tiles = [t for t, _ in info["candidates"]]
    assert tiles == [256, 512, 1024, 2048, 4096] and info["tile"] in tiles
    assert all(ms > 0 for _, ms in info["candidates"])
    for i, (a, b) in enumerate(zip(got, ref)):
        assert np.array_equal(a, b), i
    for i in (0, 2, 7):
        spec = specs[i]
        S = oracle.IndexSet.hyperbolic(spec["N"], spec["B"])
        want, _ = oracle.expmpr_propagate(S, spec, c0s[i], 0.01, 9, spec["m"])
        tol = 1e-12 if dtypes[i] == hx.HX_C128 else 1e-5
        assert np.linalg.norm(got[i] - want) / np.linalg.norm(want) <= tol, i


def test_batched_product_budget(hx):
    """A budget of 0 s: every block of a batched product stops before its first tile, flags the
    queue, and hx_batch_step returns HX_ETIMEOUT; a generous budget changes nothing."""
    specs = mixed_batch_specs()[:4]
    dtypes = [hx.HX_C64] * 4
    with pytest.raises(hx.HxError) as ei:
        run_batch(hx, specs, dtypes, nsteps=(1,), budget=0.0)
    assert ei.value.status == hx.HX_ETIMEOUT
    got, _, _ = run_batch(hx, specs, dtypes, budget=10.0)
    ref, _, _ = run_batch(hx, specs, dtypes)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


def test_batch_members_outside_batched_products(hx):
    """A member with a two-stage product (degree-8 cosine chain) keeps the batch on one graph per
    member; the step still matches the member stepped alone."""
    specs = mixed_batch_specs()[:3]
    specs[1] = dict(inputs.workload("hh2_b32"), m=7)
    specs[1]["potential"] = inputs.cos_chain(2, 0.2, 8)
    dtypes = [hx.HX_C128] * 3
    got, c0s, info = run_batch(hx, specs, dtypes)
    assert not info["batched"]
    ref, _, _ = run_batch(hx, specs, dtypes, batched="0")
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


def test_batch_schedule_autotune(hx):
    """Without HX_BATCH_BATCHED the first steps time the four schedules (one step each, across
    calls when a call has fewer steps), then the fastest runs.  The small members get the same bits
    under every schedule; the member of about a million coefficients gets the generic kernel's bits
    under the first three and, under the serial schedule, the bits of hx_step on it alone (complex64
    with fused projections: equal to the others within rounding)."""
    specs = mixed_batch_specs()[:6]
    big = dict(inputs.batch_workloads(n=1, seed=5)[0], N=3, B=20000)
    big["L"] = inputs.half_width(big["B"])
    big["potential"] = inputs.henon_heiles_chain(3, 0.1)
    big["init"] = dict(big["init"], q=[0.3, -0.2, 0.5])
    specs.append(big)
    dtypes = [hx.HX_C64] * len(specs)
    infos = []
    got, c0s, _ = run_batch(hx, specs, dtypes, nsteps=(1, 2, 6), batched=None, infos=infos)
    assert infos[0]["schedule"] == -1 and len(infos[0]["step_ms"]) == 1
    last = infos[-1]
    assert sorted(last["step_ms"]) == [hx.HX_SCHED_MEMBERS, hx.HX_SCHED_BATCHED, hx.HX_SCHED_HYBRID,
                                       hx.HX_SCHED_SERIAL]
    assert last["schedule"] == min(last["step_ms"], key=last["step_ms"].get)
    refs = {}
    for forced in ("0", "1", "2", "3"):
        refs[int(forced)], _, info = run_batch(hx, specs, dtypes, nsteps=(9,), batched=forced)
        assert info["schedule"] == int(forced)
    for sched, ref in refs.items():
        for i in range(len(specs) - 1):
            assert np.array_equal(ref[i], got[i]), (sched, i)
    for sched in (1, 2):
        assert np.array_equal(refs[sched][-1], refs[0][-1]), sched
    # the timed steps ran every schedule once, so the large member took steps of both kinds
    assert np.linalg.norm(got[-1] - refs[0][-1]) <= 1e-5 * np.linalg.norm(refs[0][-1])
    # the serial schedule's large member: hx_step on the problem alone, with its specialised kernel
    P = hx.Problem(big["N"], big["B"], dtype=hx.HX_C64, m=big["m"])
    try:
        P.set_potential(big, 0.0)
        assert hx.hx_apply_specialised(P.p) == 1
        x = torch.from_numpy(c0s[-1]).to("cuda")
        hx.hx_step(P.p, x, 0.01, 9)
        torch.cuda.synchronize()
        alone = x.cpu().numpy()
    finally:
        P.close()
    assert np.array_equal(refs[3][-1], alone)
    assert np.linalg.norm(refs[3][-1] - refs[0][-1]) <= 1e-5 * np.linalg.norm(refs[0][-1])


def _hc_size(N, B, _memo={}):
    """|{k in N^N : prod (1 + k_l) <= B}| by recursion on the first coordinate."""
    if N == 0:
        return 1
    key = (N, B)
    if key not in _memo:
        _memo[key] = sum(_hc_size(N - 1, B // (1 + k)) for k in range(B))
    return _memo[key]


def test_batch_members_of_the_256_problem_workload(hx, oracle):
    """Members of the 256-problem workload itself (N ~ U{2..8}, B log-uniform in [64, 8192]): the six
    smallest, three of about 9e4 coefficients and the two closest to 2.4 M and 3.1 M, stepped
    together in complex64 under the batched and the serial schedules.  Every member equals hx_step
    on it alone bit for bit (the generic kernel for members in the batched launches, its
    specialised kernel for a large member under the serial schedule); the two smallest match the
    oracle."""
    all_specs = inputs.batch_workloads(n=256, seed=3)
    by_size = sorted(range(len(all_specs)), key=lambda i: _hc_size(all_specs[i]["N"], all_specs[i]["B"]))
    sizes = {i: _hc_size(all_specs[i]["N"], all_specs[i]["B"]) for i in by_size}
    mid = [i for i in by_size if 8e4 < sizes[i] < 2e5][:3]
    large = [min(by_size, key=lambda i: abs(sizes[i] - t)) for t in (2.4e6, 3.1e6)]
    pick = by_size[:6] + mid + large
    specs = [all_specs[i] for i in pick]
    dtypes = [hx.HX_C64] * len(specs)
    nsteps = (2, 1)
    serial, c0s, info = run_batch(hx, specs, dtypes, nsteps=nsteps, batched="3")
    batched, _, _ = run_batch(hx, specs, dtypes, nsteps=nsteps, batched="1")
    assert info["schedule"] == hx.HX_SCHED_SERIAL
    for j, (spec, c0) in enumerate(zip(specs, c0s)):
        for generic, want in ((True, batched[j]), (j < len(specs) - 2, serial[j])):
            P = hx.Problem(spec["N"], spec["B"], dtype=hx.HX_C64, m=spec["m"])
            try:
                with env("HX_APPLY_SPECIALISE", "0" if generic else None):
                    P.set_potential(spec, 0.0)
                assert generic or hx.hx_apply_specialised(P.p) == 1
                x = torch.from_numpy(c0).to("cuda")
                hx.hx_step(P.p, x, 0.01, sum(nsteps))
                torch.cuda.synchronize()
                assert np.array_equal(x.cpu().numpy(), want), (j, generic)
            finally:
                P.close()
    for j in (0, 1):
        spec = specs[j]
        S = oracle.IndexSet.hyperbolic(spec["N"], spec["B"])
        ref, _ = oracle.expmpr_propagate(S, spec, c0s[j], 0.01, sum(nsteps), spec["m"])
        assert np.linalg.norm(serial[j] - ref) <= 1e-5 * np.linalg.norm(ref), j
