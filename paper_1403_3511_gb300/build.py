"""Builds libhx.so (the CUDA library behind include/hx.h) in-tree with nvcc for sm_103a."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libhx.so")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["hx_capi.cu", "hx_apply.cu", "hx_krylov.cu", "hx_noalloc.cu", "hx_adjoint.cu", "hx_jit.cu"]
# headers that the run-time compiler (NVRTC) gets as text, for the kernels specialised per potential
JIT_HEADERS = [("kJitTypesSource", "hx_types.h"), ("kJitStencilSource", "hx_stencil.cuh")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "-I", os.path.join(os.path.dirname(HERE), "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def cuda_home() -> str:
    path = nvcc()
    if os.path.isabs(path):
        return os.path.dirname(os.path.dirname(path))
    return os.environ.get("CUDA_HOME", "/usr/local/cuda")


def write_jit_sources() -> None:
    """The headers of the specialised kernels as C string literals (_build/hx_jit_sources.inc)."""
    out = ["// generated by build.py from " + ", ".join(f for _, f in JIT_HEADERS)]
    for var, name in JIT_HEADERS:
        text = open(os.path.join(CSRC, name)).read()
        if ")HXSRC" in text:
            raise RuntimeError(f"{name} contains the raw-string delimiter")
        out.append(f'static const char {var}[] = R"HXSRC(' + text + ')HXSRC";')
    path = os.path.join(BUILD, "hx_jit_sources.inc")
    new = "\n".join(out) + "\n"
    if not os.path.exists(path) or open(path).read() != new:
        with open(path, "w") as f:
            f.write(new)


def _newest_input() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(os.path.dirname(HERE), "include", "hx.h")]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, extra: list | None = None) -> str:
    if not force and os.path.exists(OUT) and os.path.getmtime(OUT) >= _newest_input():
        return OUT
    os.makedirs(BUILD, exist_ok=True)
    write_jit_sources()
    extra = extra or []

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc(), *ARCH, *FLAGS, "-I", BUILD, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr, file=sys.stderr)
        return obj

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = OUT + f".tmp{os.getpid()}"
    lib = os.path.join(cuda_home(), "lib64")
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-L", lib, "-lnvrtc", "-Xlinker", "-rpath=" + lib]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None))
