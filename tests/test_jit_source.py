"""The kernels compiled per potential (csrc/hx_jit.cu writes their source, NVRTC compiles it when a
potential is set) are built from templates in csrc/hx_stencil.cuh that the library's own build does
not instantiate.  This compiles a generated source (tests/native/jit_hh6_c64.cu: the N=6 Hénon-Heiles
chain of the benchmark) against the current header with nvcc for sm_103a, so that a header change that
breaks those kernels fails here rather than at run time (where the library would fall back to the
generic kernel), and checks the register budgets the launch bounds give: the single-time product
kernels in 64 registers without spills, the two-time (Magnus) kernels in 80 registers.  The same source
rewritten for complex128 states (R = double) checks the FP64 stencils the same way."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1403_3511_gb300", "csrc")


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    return None


FIXTURE = os.path.join(ROOT, "tests", "native", "jit_hh6_c64.cu")


def _complex128_source() -> str:
    """The same operator sequence as the generator writes it for complex128 states: R = double, 3 blocks
    of 256 per SM for every kernel, and without the kernels that exist for complex64 only (the
    product with fused projections or with the Rayleigh quotient)."""
    src = open(FIXTURE).read().replace("using R = float;", "using R = double;")
    for name in ("hx_apply_specialised_dots", "hx_apply_specialised_rq"):
        i = src.index(name + "(const __grid_constant__")
        start = src.rindex('extern "C"', 0, i)
        end = src.index("\n}\n", i) + 3
        src = src[:start] + src[end:]
    return src.replace("__launch_bounds__(hx::kApplyThreads, 4)", "__launch_bounds__(hx::kApplyThreads, 3)")


def _ptxas_info(path: str, cubin: str) -> dict:
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    r = subprocess.run([nvcc, "-cubin", "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O3",
                        "-I", CSRC, path, "-o", cubin, "-Xptxas", "-v"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    # per kernel: "Compiling entry function 'k'", "Function properties for k" with its stack frame and
    # spills (functions it calls get their own properties lines), "Used n registers"
    info, cur, prop = {}, None, None
    for line in r.stderr.splitlines():
        m = re.search(r"entry function '(\w+)'", line)
        if m:
            cur, prop = m.group(1), None
            info[cur] = {}
        m = re.search(r"Function properties for (\w+)", line)
        if m:
            prop = m.group(1)
        m = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m and cur is not None and prop == cur:
            info[cur]["spill"] = int(m.group(1))   # bytes of spill stores
        m = re.search(r"Used (\d+) registers", line)
        if m and cur is not None:
            info[cur]["regs"] = int(m.group(1))
    return info


OUT_DIR = os.path.join(ROOT, "paper_1403_3511_gb300", "_build")


@pytest.fixture(scope="module")
def ptxas_info():
    os.makedirs(OUT_DIR, exist_ok=True)
    return _ptxas_info(FIXTURE, os.path.join(OUT_DIR, "jit_hh6_c64.cubin"))


@pytest.fixture(scope="module")
def ptxas_info_c128():
    os.makedirs(OUT_DIR, exist_ok=True)
    path = os.path.join(OUT_DIR, "jit_hh6_c128.cu")
    with open(path, "w") as f:
        f.write(_complex128_source())
    return _ptxas_info(path, os.path.join(OUT_DIR, "jit_hh6_c128.cubin"))


def test_generated_source_compiles_with_every_kernel(ptxas_info):
    want = {"hx_apply_specialised", "hx_apply_specialised_rq", "hx_apply_specialised_dots",
            "hx_apply_specialised_dual", "hx_apply_specialised_pair", "hx_apply_tops"}
    assert want <= set(ptxas_info), sorted(ptxas_info)


@pytest.mark.parametrize("kernel", ["hx_apply_specialised", "hx_apply_specialised_rq"])
def test_single_time_products_fit_64_registers_without_spills(ptxas_info, kernel):
    k = ptxas_info[kernel]
    assert k["regs"] <= 64 and k["spill"] == 0, k


@pytest.mark.parametrize("kernel,max_spill", [("hx_apply_specialised_dual", 0), ("hx_apply_specialised_pair", 128)])
def test_two_time_products_fit_80_registers(ptxas_info, kernel, max_spill):
    k = ptxas_info[kernel]
    assert k["regs"] <= 80 and k["spill"] <= max_spill, k


def test_complex128_product_fits_80_registers_without_spills(ptxas_info_c128):
    """The FP64 plane stencils (one combined weight per footprint point) in the complex128 product."""
    assert {"hx_apply_specialised", "hx_apply_specialised_dual", "hx_apply_specialised_pair"} <= set(ptxas_info_c128)
    k = ptxas_info_c128["hx_apply_specialised"]
    assert k["regs"] <= 80 and k["spill"] == 0, k
