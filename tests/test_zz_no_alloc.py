"""hx_norm_noalloc: the norm for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc when they need a norm, for example an application whose
device memory is held by its own pool, or a latency-critical loop.  hx_norm_noalloc keeps its
reduction scratch in a fixed array inside libhx.so instead.  This file checks, through the C ABI,
that it returns what hx_norm returns, on two calls in a row (the fixed array keeps the previous
call's contents, so the second call checks that nothing stale leaks).  It is collected last and
also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_1403_3511_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL_C128 = 1e-12


@pytest.fixture(scope="module")
def hx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_3511_gb300 import build
    build.build()
    from paper_1403_3511_gb300 import hx as _hx
    return _hx


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_norm_noalloc_matches_norm(hx, dtype):
    spec = inputs.workload("hh6_b4096")
    dt = hx.HX_C128 if dtype == "c128" else hx.HX_C64
    tdt = torch.complex128 if dtype == "c128" else torch.complex64
    P = hx.Problem(spec["N"], spec["B"], dtype=dt)
    try:
        P.set_potential(spec, 0.0)
        g = torch.Generator(device="cuda").manual_seed(5)
        x = torch.randn(P.size, dtype=tdt, device="cuda", generator=g)
        y = 3.0 * torch.randn(P.size, dtype=tdt, device="cuda", generator=g)
        got = [hx.hx_norm_noalloc(P.p, x), hx.hx_norm_noalloc(P.p, y)]      # two calls in a row
        want = [hx.hx_norm(P.p, x), hx.hx_norm(P.p, y)]
        for a, b in zip(got, want):
            assert abs(a - b) <= TOL_C128 * b, (a, b)
        assert abs(hx.hx_norm_noalloc(P.p, x) - want[0]) <= TOL_C128 * want[0]
        ref = torch.linalg.vector_norm(x.to(torch.complex128)).item()
        assert abs(got[0] - ref) <= TOL_C128 * ref
    finally:
        P.close()
