"""Compile the CUDA library for sm_103a into an in-tree shared object.

Each translation unit under ``csrc/`` is compiled by nvcc in parallel and
linked into ``_build/<machine>/libfamst.so`` (the CUDA runtime is linked
statically, so the library needs only the driver at run time).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import platform
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def out_dir() -> str:
    return os.path.join(PKG, "_build", platform.machine())


def lib_path() -> str:
    return os.path.join(out_dir(), "libfamst.so")


def checked_lib_path() -> str:
    return os.path.join(out_dir(), "libfamst_checked.so")


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _nvcc() -> str:
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False) -> str:
    od = out_dir()
    os.makedirs(od, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    nvcc = _nvcc()
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                    "-I", INCLUDE, "-I", CSRC, "--expt-relaxed-constexpr"]
    if ptxas_v:
        flags += ["-Xptxas", "-v"]

    def compile_one(src: str) -> str:
        obj = os.path.join(od, os.path.basename(src)[:-3] + ".o")
        if force or ptxas_v or _stale(obj, [src] + headers):
            cmd = [nvcc, "-c", src, "-o", obj] + flags
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
            if verbose or ptxas_v:
                print(r.stderr, end="")
        return obj

    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(compile_one, srcs))
    lib = lib_path()
    _link(nvcc, lib, objs, force)
    return lib


def _link(nvcc: str, lib: str, objs: list[str], force: bool) -> None:
    if force or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "static"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)


def build_checked(force: bool = False) -> str:
    """The debug build: the C ABI compiled with FAMST_CHECK_BOUNDS (every
    index array a build stage hands to the next is validated on the device
    before use; a violation fails the call instead of faulting), linked with
    the release kernels into libfamst_checked.so beside libfamst.so."""
    build()
    od = out_dir()
    nvcc = _nvcc()
    src = os.path.join(CSRC, "famst_api.cu")
    obj = os.path.join(od, "famst_api_checked.o")
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    if force or _stale(obj, [src] + headers):
        cmd = [nvcc, "-c", src, "-o", obj, "-DFAMST_CHECK_BOUNDS"] + ARCH + [
            "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-I", INCLUDE, "-I",
            CSRC, "--expt-relaxed-constexpr"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    objs = [os.path.join(od, os.path.basename(s)[:-3] + ".o") for s in sources()
            if os.path.basename(s) != "famst_api.cu"] + [obj]
    lib = checked_lib_path()
    _link(nvcc, lib, objs, force)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, ptxas_v="-v" in sys.argv))
