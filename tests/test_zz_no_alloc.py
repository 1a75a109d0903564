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


def _cudart():
    """The CUDA runtime library of the toolkit (for the memory-pool probe below)."""
    import ctypes
    import os
    from paper_1403_3511_gb300 import build
    for name in ("libcudart.so", "libcudart.so.13"):
        path = os.path.join(build.cuda_home(), "lib64", name)
        if os.path.exists(path):
            return ctypes.CDLL(path)
    pytest.skip("no libcudart.so in the CUDA toolkit")


def test_norm_noalloc_rejects_misaligned_vector(hx):
    """A vector off its element alignment is refused on the host (HX_EINVAL), before any launch."""
    import ctypes
    spec = inputs.workload("hh2_b32")
    P = hx.Problem(spec["N"], spec["B"], dtype=hx.HX_C128)
    try:
        x = torch.zeros(P.size + 1, dtype=torch.complex128, device="cuda")
        out = ctypes.c_double()
        st = hx.lib.hx_norm_noalloc(P.p, ctypes.c_void_p(x.data_ptr() + 4), ctypes.byref(out))
        assert st == hx.HX_EINVAL, st
        assert "aligned" in hx.hx_last_error()
    finally:
        P.close()


def test_norm_noalloc_allocates_nothing(hx):
    """The device's default memory pool (where hx_norm takes its scratch with cudaMallocAsync) sees
    no allocation from hx_norm_noalloc: its high-water mark stays at the current use, and then rises
    with hx_norm, which shows that the probe detects an allocation."""
    import ctypes
    rt = _cudart()
    spec = inputs.workload("hh6_b4096")
    P = hx.Problem(spec["N"], spec["B"], dtype=hx.HX_C64)
    try:
        x = torch.randn(P.size, dtype=torch.complex64, device="cuda", generator=torch.Generator(device="cuda").manual_seed(3))
        torch.cuda.synchronize()
        pool = ctypes.c_void_p()
        assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), torch.cuda.current_device()) == 0
        used_current, used_high = 7, 8          # cudaMemPoolAttrUsedMemCurrent, cudaMemPoolAttrUsedMemHigh

        def attr(a):
            v = ctypes.c_uint64()
            assert rt.cudaMemPoolGetAttribute(pool, a, ctypes.byref(v)) == 0
            return v.value

        zero = ctypes.c_uint64(0)
        assert rt.cudaMemPoolSetAttribute(pool, used_high, ctypes.byref(zero)) == 0   # reset the mark
        base = attr(used_current)
        a = hx.hx_norm_noalloc(P.p, x)
        b = hx.hx_norm_noalloc(P.p, x)
        assert attr(used_high) <= base, (attr(used_high), base)
        c = hx.hx_norm(P.p, x)
        assert attr(used_high) > base
        assert abs(a - c) <= TOL_C128 * c and a == b
    finally:
        P.close()


def test_norm_noalloc_reports_nonfinite(hx):
    """A NaN in the vector gives HX_ENONFINITE (planted on the host before the copy)."""
    spec = inputs.workload("hh2_b32")
    P = hx.Problem(spec["N"], spec["B"], dtype=hx.HX_C128)
    try:
        c = np.ones(P.size, dtype=np.complex128)
        c[7] = np.nan
        x = torch.from_numpy(c).to("cuda")
        with pytest.raises(hx.HxError) as ei:
            hx.hx_norm_noalloc(P.p, x)
        assert ei.value.status == hx.HX_ENONFINITE
    finally:
        P.close()
