"""GPU parity of the index set and the matrix-free product against the oracle (through the C ABI)."""
import numpy as np
import pytest

from paper_1403_3511_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL_C128 = 1e-12      # FP64 path: relative to max |y_ref|
TOL_C64 = 1e-5        # complex64 stencil: relative 2-norm error


@pytest.fixture(scope="module")
def hx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_3511_gb300 import build
    build.build()
    from paper_1403_3511_gb300 import hx as _hx
    return _hx


def spec_of(N, B, potential, L=None):
    return dict(N=N, B=B, L=L or inputs.half_width(B), potential=potential)


def gpu_apply(hx, P, c):
    tdt = torch.complex64 if P.dtype == hx.HX_C64 else torch.complex128
    x = torch.from_numpy(np.ascontiguousarray(c)).to("cuda", tdt)
    y = torch.empty_like(x)
    hx.hx_apply(P.p, x, y)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.complex128)


def make(hx, spec, dtype, order="sym", t=0.0):
    P = hx.Problem(spec["N"], spec["B"], dtype=dtype, order=order)
    P.set_potential(spec, t)
    return P


@pytest.mark.parametrize("N,B", [(1, 1), (1, 50), (2, 1), (2, 32), (3, 100), (4, 512), (6, 300), (10, 64), (7, 2000)])
def test_export_rank_unrank_bit_exact(hx, oracle, N, B):
    S = oracle.IndexSet.hyperbolic(N, B)
    s = hx.hx_indexset_create(N, B)
    try:
        assert hx.hx_indexset_size(s) == S.size
        k = hx.hx_indexset_export(s, N)
        assert np.array_equal(k, S.k)
        for i in inputs.sample_rows(S.size, 50):
            assert hx.hx_indexset_rank(s, S.k[i]) == i
            assert np.array_equal(hx.hx_indexset_unrank(s, int(i), N), S.k[i])
        assert hx.hx_indexset_rank(s, np.full(N, B)) == -1
    finally:
        hx.hx_indexset_destroy(s)


def random_spec(rng, N, B, nterms, maxdeg):
    comps = []
    for _ in range(nterms):
        axes = sorted(rng.choice(N, size=min(N, rng.integers(1, 3)), replace=False).tolist())
        powers = {int(a): int(rng.integers(1, maxdeg + 1)) for a in axes}
        comps.append({"coef": float(rng.standard_normal()), "powers": powers})
    return spec_of(N, B, comps)


CASES = {
    "hh2_b32": lambda: inputs.workload("hh2_b32"),
    "hh3_b300_dipole": lambda: spec_of(3, 300, inputs.henon_heiles_chain(3, 0.111, (0.05, 1.0))),
    "ctrl4_b512": lambda: inputs.workload("ctrl4_b512"),
    "cos3_b64": lambda: spec_of(3, 64, inputs.cos_chain(3, 0.2, 8)),
    "cos4_b40_deg5": lambda: spec_of(4, 40, inputs.cos_chain(4, 0.3, 5)),
    "line1_b50": lambda: spec_of(1, 50, [{"coef": 0.3, "powers": {0: 3}}, {"coef": -0.2, "powers": {0: 1}}]),
    "rand5_b150": lambda: random_spec(np.random.default_rng(11), 5, 150, 8, 3),
    "rand4_b90_deg6": lambda: random_spec(np.random.default_rng(12), 4, 90, 5, 6),
    "hh6_b2000": lambda: spec_of(6, 2000, inputs.henon_heiles_chain(6, 0.111, (0.05, 1.0))),
    # rows longer than 2^15 (the first row holds B elements)
    "hh2_b40000": lambda: spec_of(2, 40000, inputs.henon_heiles_chain(2, 0.111, (0.05, 1.0))),
    # line ops on the second axis of plane ops: merged with a (2,1) op at degree 3 and with a (2,2)
    # op at degree 2; they stay separate beside a (3,1) plane op, whose stencil is not specialised,
    # and beside a (1,1) plane op, whose stencil never visits the points s = 0 of a merged line
    "merge4_b160": lambda: spec_of(4, 160, [
        {"coef": 0.11, "powers": {0: 2, 1: 1}}, {"coef": -0.04, "powers": {1: 3}},
        {"coef": 0.07, "powers": {1: 2, 2: 2}}, {"coef": 0.05, "powers": {2: 2}},
        {"coef": 0.09, "powers": {0: 3, 3: 1}}, {"coef": 0.03, "powers": {3: 3}},
        {"coef": -0.02, "powers": {2: 1, 3: 1}}, {"coef": 0.06, "powers": {3: 1}}]),
}


def check(y, ref, dtype, hx, bound=None):
    """FP64: max-abs error relative to max |y_ref|, or, for potentials whose Chebyshev terms cancel,
    the normwise bound eps * (max D + sum |alpha|) * ||c|| of evaluating the expansion term by term
    (each product of T_r(X/L) has 2-norm <= 1 because L exceeds the spectral radius of every fibre)."""
    if dtype == hx.HX_C128 and bound is not None:
        err = np.linalg.norm(y - ref)
        assert err <= TOL_C128 * bound, (err, bound)
    elif dtype == hx.HX_C128:
        err = np.abs(y - ref).max() / np.abs(ref).max()
        assert err <= TOL_C128, err
    else:
        err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
        assert err <= TOL_C64, err


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_apply_matches_oracle(hx, oracle, case, dtype):
    spec = CASES[case]()
    dt = hx.HX_C128 if dtype == "c128" else hx.HX_C64
    t = 0.7
    S = oracle.IndexSet.hyperbolic(spec["N"], spec["B"])
    c = inputs.initial_vector({"init": {"kind": "gaussian", "seed": 5}}, S.k)
    r, a = oracle.potential_terms(spec, t)
    ref = oracle.apply(S, r, a, spec["L"], c)
    bound = (oracle.diag(S).max() + np.abs(a).sum()) * np.linalg.norm(c) if case.startswith(("rand", "merge")) else None
    P = make(hx, spec, dt, t=t)
    try:
        y = gpu_apply(hx, P, c)
        check(y, ref, dt, hx, bound)
        if bound is not None and dt == hx.HX_C128:
            # beside the normwise bound, the max-abs error relative to max |y_ref|: the Chebyshev
            # terms of these random potentials cancel (sum |alpha| / max |y| up to about 1e5), so
            # the attainable accuracy is 1e-16 times that ratio; two term orders of the oracle
            # itself differ by up to 7.5e-10 relative
            err = np.abs(y - ref).max() / np.abs(ref).max()
            assert err <= 2e-9, err
    finally:
        P.close()


@pytest.mark.parametrize("order", ["eq", "alg"])
def test_literal_orders_match_oracle(hx, oracle, order):
    spec = random_spec(np.random.default_rng(3), 4, 200, 7, 3)
    S = oracle.IndexSet.hyperbolic(4, 200)
    c = inputs.initial_vector({"init": {"kind": "gaussian", "seed": 6}}, S.k)
    r, a = oracle.potential_terms(spec, 0.0)
    ref = oracle.apply(S, r, a, spec["L"], c, order)
    P = make(hx, spec, hx.HX_C128, order=order)
    try:
        check(gpu_apply(hx, P, c), ref, hx.HX_C128, hx)
    finally:
        P.close()


@pytest.mark.parametrize("name", ["hh6_b4096", "cos10_b1024"])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_full_size_sampled_rows(hx, oracle, name, dtype):
    """The full-size workloads, launched exactly as the benchmark does, checked on sampled rows
    that the oracle computes one at a time (first and last rows included)."""
    spec = inputs.workload(name)
    dt = hx.HX_C128 if dtype == "c128" else hx.HX_C64
    S = oracle.IndexSet.hyperbolic(spec["N"], spec["B"])
    c = inputs.initial_vector(spec, S.k)
    t = 0.25
    r, a = oracle.potential_terms(spec, t)
    rows = inputs.sample_rows(S.size, 400, seed=9)
    ref = oracle.apply_rows(S, spec["B"], r, a, spec["L"], c, rows)
    P = make(hx, spec, dt, t=t)
    try:
        y = gpu_apply(hx, P, c)
    finally:
        P.close()
    tol = TOL_C128 if dt == hx.HX_C128 else TOL_C64
    err = np.abs(y[rows] - ref).max() / np.abs(ref).max()
    assert err <= tol, err


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_full_size_every_element(hx, oracle, dtype):
    """The N = 6, B = 4096 Henon-Heiles chain with its dipole (4,883,360 coefficients), launched as
    the benchmark does, against the oracle's full product, element by element."""
    spec = inputs.workload("hh6_b4096")
    dt = hx.HX_C128 if dtype == "c128" else hx.HX_C64
    S = oracle.IndexSet.hyperbolic(spec["N"], spec["B"])
    c = inputs.initial_vector(spec, S.k)
    t = 0.25
    r, a = oracle.potential_terms(spec, t)
    ref = oracle.apply(S, r, a, spec["L"], c)
    P = make(hx, spec, dt, t=t)
    try:
        y = gpu_apply(hx, P, c)
    finally:
        P.close()
    if dt == hx.HX_C128:
        err = np.abs(y - ref).max() / np.abs(ref).max()
        assert err <= TOL_C128, err
    else:
        err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
        assert err <= TOL_C64, err
        # and no single element far off: each within 1e-5 of the largest output
        assert np.abs(y - ref).max() / np.abs(ref).max() <= TOL_C64


def test_edge_cases(hx, oracle):
    # single element, no terms: A = D
    P = hx.Problem(3, 1)
    try:
        hx.hx_potential_set(P.p, 5.0, [], 0.0)
        y = gpu_apply(hx, P, np.array([2.0 + 1.0j]))
        assert np.allclose(y, [1.5 * (2.0 + 1.0j)], atol=0)
    finally:
        P.close()
    # constant term folds into the diagonal; a term on the last axis only
    spec = spec_of(2, 20, [{"coef": 0.4, "powers": {}}, {"coef": 0.7, "powers": {1: 2}}])
    S = oracle.IndexSet.hyperbolic(2, 20)
    c = inputs.initial_vector({"init": {"kind": "gaussian", "seed": 1}}, S.k)
    r, a = oracle.potential_terms(spec, 0.0)
    P = make(hx, spec, hx.HX_C128)
    try:
        check(gpu_apply(hx, P, c), oracle.apply(S, r, a, spec["L"], c), hx.HX_C128, hx)
    finally:
        P.close()


def test_time_modulation_and_set_time(hx, oracle):
    spec = inputs.workload("ctrl4_b512")
    S = oracle.IndexSet.hyperbolic(4, 512)
    c = inputs.initial_vector({"init": {"kind": "gaussian", "seed": 2}}, S.k)
    P = make(hx, spec, hx.HX_C128, t=0.0)
    try:
        for t in (0.0, 0.05, 0.049999, 3.3, 9.99, 10.0, 12.0):   # interval edges and outside [0, T)
            hx.hx_set_time(P.p, t)
            assert hx.hx_get_time(P.p) == t
            r, a = oracle.potential_terms(spec, t)
            check(gpu_apply(hx, P, c), oracle.apply(S, r, a, spec["L"], c), hx.HX_C128, hx)
    finally:
        P.close()


def test_deterministic(hx):
    spec = inputs.workload("hh6_b4096")
    P = make(hx, spec, hx.HX_C64)
    try:
        x = torch.randn(P.size, dtype=torch.complex64, device="cuda")
        y1, y2 = torch.empty_like(x), torch.empty_like(x)
        hx.hx_apply(P.p, x, y1)
        hx.hx_apply(P.p, x, y2)
        torch.cuda.synchronize()
        assert torch.equal(y1, y2)
    finally:
        P.close()


def test_host_entry_point(hx, oracle):
    spec = inputs.workload("hh2_b32")
    S = oracle.IndexSet.hyperbolic(2, 32)
    c = inputs.initial_vector(spec, S.k)
    P = make(hx, spec, hx.HX_C128)
    try:
        out = np.zeros_like(c)
        hx.hx_apply_host(P.p, c, out)
        r, a = oracle.potential_terms(spec, 0.0)
        check(out, oracle.apply(S, r, a, spec["L"], c), hx.HX_C128, hx)
    finally:
        P.close()


def test_errors(hx):
    P = hx.Problem(3, 20)
    try:
        x = torch.zeros(P.size, dtype=torch.complex128, device="cuda")
        with pytest.raises(hx.HxError):
            hx.hx_apply(P.p, x, torch.empty_like(x))          # no potential yet
        with pytest.raises(hx.HxError) as ei:
            hx.hx_potential_set(P.p, 5.0, [{"axes": [0, 1, 2], "coef": np.ones((2, 2, 2))}], 0.0)
        assert ei.value.status in (-1, -7)
        with pytest.raises(hx.HxError):
            hx.hx_potential_set(P.p, -1.0, [], 0.0)
        with pytest.raises(hx.HxError):
            hx.hx_potential_set(P.p, 5.0, [{"axes": [1, 0], "coef": np.ones((2, 2))}], 0.0)
    finally:
        P.close()


@pytest.mark.parametrize("case", ["hh6_b2000", "ctrl4_b512", "hh3_b300_dipole", "hh2_b40000", "cos3_b64"])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_specialised_kernel_matches_generic(hx, case, dtype, monkeypatch):
    """Potentials whose operators all have specialised stencils run a kernel compiled for their
    operator sequence at hx_potential_set; it computes what the generic kernel computes (the cosine
    chain: degree-8 line operators and a compiled channel stage)."""
    spec = CASES[case]()
    dt = hx.HX_C128 if dtype == "c128" else hx.HX_C64
    n = None
    outs = []
    for flag in ("1", "0"):
        monkeypatch.setenv("HX_APPLY_SPECIALISE", flag)
        P = make(hx, spec, dt, t=0.3)
        try:
            assert hx.hx_apply_specialised(P.p) == (1 if flag == "1" else 0), hx.hx_last_error()
            if n is None:
                n = P.size
                c = inputs.complex_gaussian(n, 4)
            outs.append(gpu_apply(hx, P, c))
        finally:
            P.close()
    err = np.abs(outs[0] - outs[1]).max() / np.abs(outs[1]).max()
    assert err <= (1e-14 if dtype == "c128" else 1e-6), err


@pytest.mark.parametrize("case,why", [("merge4_b160", "no specialised stencil"), ("rand4_b90_deg6", "no specialised stencil"),
                                      ("cos4_b40_deg5", "no specialised stencil")])
def test_potentials_without_specialised_kernel(hx, case, why):
    """Plane operators of degree 3 or more keep the generic kernel."""
    P = make(hx, CASES[case](), hx.HX_C64)
    try:
        assert hx.hx_apply_specialised(P.p) == 0
        assert why in hx.hx_last_error()
    finally:
        P.close()


@pytest.mark.parametrize("case,dtype,k,fused", [
    ("hh3_b300_dipole", "c64", 0, True), ("hh3_b300_dipole", "c64", 3, True), ("hh3_b300_dipole", "c64", 7, True),
    ("hh6_b2000", "c64", 5, True), ("hh2_b40000", "c64", 2, True),
    ("hh3_b300_dipole", "c128", 4, False), ("cos3_b64", "c64", 6, False), ("cos3_b64", "c128", 7, False)])
def test_apply_project_matches_oracle(hx, oracle, case, dtype, k, fused):
    """hx_apply_project: the product against the oracle and h_i = <basis_i, y> against FP64 sums of
    the returned y, in one kernel (specialised complex64 kernels) or with a projection kernel after
    the product.  The basis holds the input itself, random vectors and a row stride above |K|."""
    spec = CASES[case]()
    dt = hx.HX_C128 if dtype == "c128" else hx.HX_C64
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    S = oracle.IndexSet.hyperbolic(spec["N"], spec["B"])
    n = S.size
    c = inputs.initial_vector({"init": {"kind": "gaussian", "seed": 8}}, S.k)
    basis_np = np.stack([c] + [inputs.complex_gaussian(n, 20 + i) / np.sqrt(2 * n) for i in range(k)])
    r, a = oracle.potential_terms(spec, 0.4)
    ref = oracle.apply(S, r, a, spec["L"], c)
    P = make(hx, spec, dt, t=0.4)
    try:
        assert bool(hx.hx_apply_specialised(P.p) and dtype == "c64" and hx.hx_step_launches(P.p)[0] == 1) == fused
        basis = torch.zeros((k + 1, n + 37), dtype=tdt, device="cuda")[:, :n]
        basis.copy_(torch.from_numpy(basis_np).to(tdt))
        x = basis[0].clone()
        y = torch.empty_like(x)
        h = torch.full((2 * (k + 1),), float("nan"), dtype=torch.float64, device="cuda")
        hx.hx_apply_project(P.p, x, y, basis, k, h)
        torch.cuda.synchronize()
        yg = y.cpu().numpy().astype(np.complex128)
        check(yg, ref, dt, hx)
        bg = basis.cpu().numpy().astype(np.complex128)
        href = bg.conj() @ yg
        got = h.cpu().numpy()
        got = got[0::2] + 1j * got[1::2]
        scale = np.linalg.norm(bg, axis=1) * np.linalg.norm(yg)
        tol = 1e-13 if dtype == "c128" else 1e-6
        assert np.all(np.abs(got - href) <= tol * scale), (np.abs(got - href) / scale).max()
    finally:
        P.close()


def test_apply_project_argument_errors(hx):
    spec = CASES["hh2_b32"]()
    P = make(hx, spec, hx.HX_C64)
    try:
        x = torch.zeros(P.size, dtype=torch.complex64, device="cuda")
        y = torch.empty_like(x)
        basis = torch.zeros((9, P.size), dtype=torch.complex64, device="cuda")
        h = torch.zeros(18, dtype=torch.float64, device="cuda")
        for kk in (-1, 8):
            with pytest.raises(hx.HxError):
                hx.hx_apply_project(P.p, x, y, basis, kk, h)
        with pytest.raises(hx.HxError):
            hx.hx_apply_project(P.p, x, x, basis, 0, h)
        with pytest.raises(hx.HxError):          # row stride below |K|
            hx.hx_apply_project(P.p, x, y, basis.view(-1)[: 2 * (P.size - 1)].view(2, P.size - 1), 1, h)
        # pointers off the element alignment are refused on the host (nothing is launched)
        import ctypes
        bad = ctypes.c_void_p(x.data_ptr() + 4)
        assert hx.lib.hx_apply(P.p, bad, ctypes.c_void_p(y.data_ptr())) == hx.HX_EINVAL
        assert hx.lib.hx_apply_project(P.p, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                       ctypes.c_void_p(basis.data_ptr() + 4), P.size, 0,
                                       ctypes.c_void_p(h.data_ptr())) == hx.HX_EINVAL
        assert hx.lib.hx_step(P.p, ctypes.c_void_p(h.data_ptr() + 8), 0.01, 1) == hx.HX_EINVAL
        # overlapping vectors are refused on the host: one shared element is enough
        buf = torch.zeros(2 * P.size - 1, dtype=torch.complex64, device="cuda")
        with pytest.raises(hx.HxError):
            hx.hx_apply(P.p, buf[: P.size], buf[P.size - 1:])
        with pytest.raises(hx.HxError):          # y is a basis vector the projections read
            hx.hx_apply_project(P.p, x, basis[1], basis, 1, h)
        hx.hx_apply_project(P.p, basis[1], y, basis, 1, h)   # c may be a basis vector
        hx.hx_apply(P.p, buf[: P.size], torch.empty_like(x))
        torch.cuda.synchronize()
    finally:
        P.close()


@pytest.mark.parametrize("dtype,specialise,offset", [("c64", True, 0), ("c64", True, 1), ("c64", False, 0),
                                                     ("c64", False, 1), ("c128", True, 0)])
def test_apply_rayleigh_matches_oracle(hx, oracle, dtype, specialise, offset, monkeypatch):
    """hx_apply_rayleigh: y = A c and r = <c, y> against the oracle, with the product kernel that
    computes r itself (complex64, specialised), with the product and the reduction kernel, and on
    vectors starting 8 bytes off a 16-byte boundary (offset 1 element, complex64)."""
    N, B = 3, 200
    spec = dict(N=N, B=B, L=inputs.half_width(B), potential=inputs.henon_heiles_chain(N, 0.111, (0.05, 1.0)))
    S = oracle.IndexSet.hyperbolic(N, B)
    c = inputs.initial_vector({"init": {"kind": "gaussian", "seed": 12}}, S.k)
    r_, a_ = oracle.potential_terms(spec, 0.3)
    ref = oracle.apply(S, r_, a_, spec["L"], c)
    dt = hx.HX_C64 if dtype == "c64" else hx.HX_C128
    if not specialise:
        monkeypatch.setenv("HX_APPLY_SPECIALISE", "0")
    P = make(hx, spec, dt, t=0.3)
    try:
        assert hx.hx_apply_specialised(P.p) == (1 if specialise else 0)
        tdt = torch.complex64 if dt == hx.HX_C64 else torch.complex128
        buf = torch.zeros(2 * (S.size + 2), dtype=tdt, device="cuda")
        x = buf[offset: offset + S.size]
        y = buf[S.size + 2 + offset: S.size + 2 + offset + S.size]
        x.copy_(torch.from_numpy(c).to(tdt))
        r = torch.zeros(2, dtype=torch.float64, device="cuda")
        hx.hx_apply_rayleigh(P.p, x, y, r)
        torch.cuda.synchronize()
        yy = y.cpu().numpy().astype(np.complex128)
        cc = x.cpu().numpy().astype(np.complex128)
        want = np.vdot(cc, ref)
        got = complex(*r.cpu().numpy())
        scale = np.linalg.norm(cc) * np.linalg.norm(ref)
        tol = 1e-12 if dt == hx.HX_C128 else 1e-5
        assert np.linalg.norm(yy - ref) <= tol * np.linalg.norm(ref)
        assert abs(got - want) <= tol * scale, (got, want)
        assert abs(hx.hx_energy(P.p, x) - want.real) <= tol * scale
        with pytest.raises(hx.HxError):                 # r inside y
            hx.hx_apply_rayleigh(P.p, x, y, y.view(torch.float64)[:2])
    finally:
        P.close()
