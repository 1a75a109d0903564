"""General downward-closed index sets and the scaled basis phi_k(S x) (Sec. 1.2, Sec. 1.4) on the
GPU, through the C ABI, against the oracle built from the same list of multi-indices."""
import numpy as np
import pytest

from paper_1403_3511_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL_C128 = 1e-12
TOL_C64 = 1e-5


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


SETS = {
    "total_degree_n4_k8": lambda: inputs.total_degree_set(4, 8),
    "random_n3_600": lambda: inputs.random_downward_closed_set(3, 600, seed=8),
    "random_n5_1500": lambda: inputs.random_downward_closed_set(5, 1500, seed=21),
}

POTENTIALS = {
    # Henon-Heiles chain with its dipole: plane operators of degrees (2, 1), cubic lines
    "hh": lambda N: inputs.henon_heiles_chain(N, 0.111, (0.05, 1.0)),
    # degree-8 cosine chain: two-stage terms through channel vectors
    "cos": lambda N: inputs.cos_chain(N, 0.2, 8),
}


def make_set(hx, ks, shuffle_seed=None):
    """The library's set from the list (optionally shuffled: the library sorts it)."""
    ks = np.array(ks)
    if shuffle_seed is not None:
        ks = ks[np.random.default_rng(shuffle_seed).permutation(len(ks))]
    return hx.hx_indexset_create_list(ks)


def gpu_apply(hx, P, c):
    tdt = torch.complex64 if P.dtype == hx.HX_C64 else torch.complex128
    x = torch.from_numpy(np.ascontiguousarray(c)).to("cuda", tdt)
    y = torch.empty_like(x)
    hx.hx_apply(P.p, x, y)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.complex128)


def check(y, ref, dtype, hx):
    if dtype == hx.HX_C128:
        err = np.abs(y - ref).max() / np.abs(ref).max()
        assert err <= TOL_C128, err
    else:
        err = rel(y, ref)
        assert err <= TOL_C64, err


@pytest.mark.parametrize("name", sorted(SETS))
def test_list_set_export_rank_unrank(hx, oracle, name):
    ks = SETS[name]()
    S = oracle.IndexSet.from_list(ks)
    s = make_set(hx, ks, shuffle_seed=3)
    try:
        N = ks.shape[1]
        assert hx.hx_indexset_size(s) == S.size
        assert np.array_equal(hx.hx_indexset_export(s, N), S.k)
        for i in inputs.sample_rows(S.size, 60):
            assert hx.hx_indexset_rank(s, S.k[i]) == i
            assert np.array_equal(hx.hx_indexset_unrank(s, int(i), N), S.k[i])
        assert hx.hx_indexset_rank(s, np.full(N, 1000)) == -1
    finally:
        hx.hx_indexset_destroy(s)


@pytest.mark.parametrize("pot", sorted(POTENTIALS))
@pytest.mark.parametrize("name", sorted(SETS))
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_list_set_apply_matches_oracle(hx, oracle, name, pot, dtype):
    ks = SETS[name]()
    N = ks.shape[1]
    S = oracle.IndexSet.from_list(ks)
    spec = dict(N=N, L=2.0 * np.sqrt(2.0 * (int(ks.max()) + 1)) + 1.0, potential=POTENTIALS[pot](N))
    t = 0.4
    r, a = oracle.potential_terms(spec, t)
    c = inputs.initial_vector({"init": {"kind": "gaussian", "seed": 6}}, S.k)
    ref = oracle.apply(S, r, a, spec["L"], c)
    dt = hx.HX_C128 if dtype == "c128" else hx.HX_C64
    s = make_set(hx, ks)
    P = hx.Problem(N, 0, dtype=dt, indexset=s)
    try:
        P.set_potential(spec, t)
        assert hx.hx_apply_specialised(P.p) == 0          # general sets run the generic kernel
        check(gpu_apply(hx, P, c), ref, dt, hx)
    finally:
        P.close()
        hx.hx_indexset_destroy(s)


def test_hyperbolic_cross_as_list_equals_hyperbolic_path(hx, oracle):
    """The hyperbolic cross given as a list runs the general-set kernel; it must give the hyperbolic
    path's product (to rounding) and the oracle's."""
    N, B = 4, 300
    S = oracle.IndexSet.hyperbolic(N, B)
    spec = dict(N=N, B=B, L=inputs.half_width(B), potential=inputs.henon_heiles_chain(N, 0.111, (0.05, 1.0)))
    c = inputs.initial_vector({"init": {"kind": "gaussian", "seed": 2}}, S.k)
    s = make_set(hx, S.k, shuffle_seed=1)
    Pl = hx.Problem(N, 0, dtype=hx.HX_C128, indexset=s)
    Ph = hx.Problem(N, B, dtype=hx.HX_C128)
    try:
        Pl.set_potential(spec, 0.2)
        Ph.set_potential(spec, 0.2)
        yl, yh = gpu_apply(hx, Pl, c), gpu_apply(hx, Ph, c)
        r, a = oracle.potential_terms(spec, 0.2)
        check(yl, oracle.apply(S, r, a, spec["L"], c), hx.HX_C128, hx)
        assert np.abs(yl - yh).max() <= 1e-13 * np.abs(yh).max()
    finally:
        Pl.close()
        Ph.close()
        hx.hx_indexset_destroy(s)


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-12), ("c64", 1e-5)])
def test_list_set_steps_match_oracle(hx, oracle, dtype, tol):
    ks = inputs.total_degree_set(4, 8)
    S = oracle.IndexSet.from_list(ks)
    spec = dict(N=4, L=9.0, potential=inputs.henon_heiles_chain(4, 0.111, (0.05, 1.0)))
    c0 = inputs.initial_vector({"init": {"kind": "coherent", "q": [0.5, -0.3, 0.8, 0.1], "eps": 1e-3, "seed": 3}}, S.k)
    ref, _ = oracle.expmpr_propagate(S, spec, c0, 0.02, 10, 7)
    s = make_set(hx, ks)
    P = hx.Problem(4, 0, dtype=hx.HX_C128 if dtype == "c128" else hx.HX_C64, indexset=s)
    try:
        P.set_potential(spec, 0.0)
        x = torch.from_numpy(c0.copy()).to("cuda")
        hx.hx_step(P.p, x, 0.02, 10)
        assert rel(x.cpu().numpy(), ref) <= tol, rel(x.cpu().numpy(), ref)
    finally:
        P.close()
        hx.hx_indexset_destroy(s)


def test_list_set_errors(hx):
    """Not downward closed, a duplicate, a negative coordinate: HX_EINVAL, nothing created."""
    bad = [np.array([[0, 0], [0, 1], [1, 1]]),          # (1, 0) missing below (1, 1)
           np.array([[0, 0], [0, 1], [0, 1]]),
           np.array([[0, 0], [0, -1]])]
    for ks in bad:
        with pytest.raises(hx.HxError) as ei:
            hx.hx_indexset_create_list(ks)
        assert ei.value.status == hx.HX_EINVAL


@pytest.mark.parametrize("scale", [0.8, 1.3])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_scaled_basis_apply_and_step(hx, oracle, scale, dtype):
    """The basis phi_k(S x): A = S^2 D_K + (1/S^2 - S^2)/2 sum X_l^2 + W(X / S), product and five
    steps against the oracle with the same S."""
    N, B = 3, 200
    S = oracle.IndexSet.hyperbolic(N, B)
    spec = dict(N=N, B=B, L=inputs.half_width(B), scale=scale,
                potential=inputs.henon_heiles_chain(N, 0.111, (0.05, 1.0)))
    dt = hx.HX_C128 if dtype == "c128" else hx.HX_C64
    c = inputs.initial_vector({"init": {"kind": "gaussian", "seed": 7}}, S.k)
    r, a = oracle.potential_terms(spec, 0.1)
    P = hx.Problem(N, B, dtype=dt, scale=scale)
    try:
        P.set_potential(spec, 0.1)
        check(gpu_apply(hx, P, c), oracle.apply(S, r, a, spec["L"], c, scale=scale), dt, hx)
        c0 = inputs.initial_vector({"init": {"kind": "coherent", "q": [0.4, 0.2, -0.5], "eps": 1e-3, "seed": 1}}, S.k)
        ref, _ = oracle.expmpr_propagate(S, spec, c0, 0.01, 5, 7, t0=0.1)
        x = torch.from_numpy(c0.copy()).to("cuda")
        hx.hx_step(P.p, x, 0.01, 5)
        assert rel(x.cpu().numpy(), ref) <= (1e-12 if dtype == "c128" else 1e-5), rel(x.cpu().numpy(), ref)
    finally:
        P.close()
