"""The C-ABI library builds, loads and exports every entry point include/hx.h declares; host-only
helpers agree with the oracle.  No GPU needed (no device call is made)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "hx.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*HX_API\s+(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(hx_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libhx():
    from paper_1403_3511_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["hx_indexset_create", "hx_potential_set", "hx_apply", "hx_step", "hx_last_error"]:
        assert required in names
    assert len(names) >= 20


def test_every_declared_symbol_is_exported(libhx):
    missing = [n for n in declared_functions() if not hasattr(libhx, n)]
    assert not missing, missing


def test_no_internal_symbols_leak(libhx):
    for n in ["build_host_tables", "launch_apply", "krylov_step"]:
        assert not hasattr(libhx, n)


def test_binding_loads_and_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1403_3511_gb300 import hx
    assert os.path.exists(hx.LIB_PATH)
    monkeypatch.setattr(hx, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        hx._load()


def test_cheb_helpers_match_oracle(oracle):
    from paper_1403_3511_gb300 import hx
    for R in (3, 8):
        assert np.allclose(hx.hx_cheb_nodes(R), oracle.cheb_nodes(R), atol=1e-15)
        u = oracle.cheb_nodes(R)
        v1 = np.cos(3.0 * u) + u ** 3
        assert np.allclose(hx.hx_cheb_coeffs(R, v1), oracle.cheb_coeffs_1d(v1), atol=1e-14)
        v2 = np.cos(np.subtract.outer(2.0 * u, 1.5 * u))
        assert np.allclose(hx.hx_cheb_coeffs(R, v2), oracle.cheb_coeffs_2d(v2), atol=1e-14)
    for p in range(7):
        L = 3.7
        u = oracle.cheb_nodes(p)
        assert np.allclose(hx.hx_cheb_monomial(p, L), oracle.cheb_coeffs_1d((L * u) ** p), atol=1e-12 * L ** p)


def test_argument_errors_without_device(libhx):
    from paper_1403_3511_gb300 import hx
    with pytest.raises(hx.HxError):
        hx.hx_indexset_create(0, 10)
    with pytest.raises(hx.HxError):
        hx.hx_indexset_create(3, 70000)
    assert "B = 70000" in hx.hx_last_error()
    with pytest.raises(hx.HxError):
        hx.hx_cheb_nodes(-1)
    with pytest.raises(hx.HxError):
        hx.hx_step_launches(None)
    assert "NULL problem" in hx.hx_last_error()
    assert hx.lib.hx_apply_project(None, None, None, None, 0, 0, None) == hx.HX_EINVAL
    assert "NULL argument" in hx.hx_last_error()
    assert hx.lib.hx_apply_rayleigh(None, None, None, None) == hx.HX_EINVAL
    assert "NULL argument" in hx.hx_last_error()
    assert hx.lib.hx_batch_set_budget(None, 1.0) == hx.HX_EINVAL
    assert hx.lib.hx_batch_info(None, None) == hx.HX_EINVAL
    # host vectors the library would read or write past their end are refused by the binding
    with pytest.raises(ValueError):
        hx.hx_step_host(None, np.zeros(4, np.complex64), 0.01, 1)       # the state is complex128
    with pytest.raises(ValueError):
        hx.hx_step_host(None, np.zeros(8, np.complex128)[::2], 0.01, 1)  # strided
    with pytest.raises(ValueError):
        hx.hx_apply_host(None, np.zeros(4, np.complex128), np.zeros(4, np.complex64))
    assert hx.lib.hx_step_host(None, None, 0.01, 1) == hx.HX_EINVAL


def test_config_layout_matches_header(libhx):
    """The binding's hx_config has the header's fields in the header's order."""
    import re
    from paper_1403_3511_gb300 import hx
    hdr = open(os.path.join(ROOT, "include", "hx.h")).read()
    body = re.search(r"typedef struct \{([^}]*)\} hx_config;", hdr).group(1)
    names = re.findall(r"\b(\w+);", body)
    assert names == [f[0] for f in hx.hx_config._fields_]
    with pytest.raises(hx.HxError):
        hx.hx_apply_specialised(None)


def test_struct_layouts_match_header(tmp_path):
    """hx_config and hx_batch_stats: the binding's field names follow the header's, and every
    offset and the size agree with what a C compiler makes of the header."""
    import re
    import shutil
    import subprocess
    from paper_1403_3511_gb300 import hx
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    hdr = open(os.path.join(ROOT, "include", "hx.h")).read()
    lines = []
    for cname, cls in (("hx_config", hx.hx_config), ("hx_batch_stats", hx.BatchStats)):
        body = re.search(r"typedef struct \{([^}]*)\} " + cname + ";", hdr).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        names = re.findall(r"(\w+)(?:\[\d+\])?;", body)
        assert names == [f[0] for f in cls._fields_], cname
        for f in names:
            lines.append(f'printf("%zu\\n", offsetof({cname}, {f}));')
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
    src = tmp_path / "layout.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"hx.h\"\nint main(void){" + "".join(lines) +
                   "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = []
    for cls in (hx.hx_config, hx.BatchStats):
        want += [getattr(cls, f[0]).offset for f in cls._fields_] + [ctypes.sizeof(cls)]
    assert got == want


def test_integer_float_conversions_match_host():
    """The binary64 <-> binary32 conversions that the complex64 Krylov kernels do with integer
    operations (csrc/hx_convert.h) agree bit for bit with the host's IEEE conversions."""
    import shutil
    import subprocess
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out_dir = os.path.join(ROOT, "paper_1403_3511_gb300", "_build")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "convert_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_1403_3511_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "native", "convert_check.cpp"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
