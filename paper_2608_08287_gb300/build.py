"""Build libtsdf.so in-tree with nvcc for sm_103a (GB300).

The translation units (host runtime, batches, serving, streaming host input,
tuning, and the kernels, split in two) compile in parallel, then link into
``paper_2608_08287_gb300/_build/libtsdf.so`` against the shared CUDA runtime
(so the library and PyTorch share one runtime and one context).
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libtsdf.so")
# The checked build (-DTSDF_CHECKED): every pool, table, coordinate and image
# index range-checked before use (csrc/tsdf_check.h), in a library of its own.
BUILD_CHECKED = os.path.join(BUILD, "checked")
LIB_CHECKED = os.path.join(BUILD_CHECKED, "libtsdf.so")

SOURCES = ("tsdf_api.cu", "tsdf_batch.cu", "tsdf_kernels.cu", "tsdf_kernels_split.cu",
           "tsdf_noalloc.cu", "tsdf_serve.cu", "tsdf_stream.cu", "tsdf_tune.cu")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Host code is compiled with contraction off: the per-frame constants the
# kernels' decisions depend on are computed in a fixed order of IEEE
# single-precision operations.
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler",
              "-ffp-contract=off", "-Xptxas", "-warn-spills", "--expt-relaxed-constexpr"]


def nvcc_path() -> str:
    p = shutil.which("nvcc")
    if p:
        return p
    p = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(p):
        return p
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtsdf")


def _deps():
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC)
           if f.endswith((".cu", ".cuh", ".h"))]
    out.append(os.path.join(INCLUDE, "tsdf.h"))
    return out


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build_library(force: bool = False, verbose: bool = False, extra_flags=(),
                  checked: bool = False) -> str:
    """Compile and link libtsdf.so if any source is newer than it. Returns its
    path. checked=True builds the checked library (LIB_CHECKED) instead."""
    out_dir = BUILD_CHECKED if checked else BUILD
    lib_path = LIB_CHECKED if checked else LIB
    if checked:
        extra_flags = (*extra_flags, "-DTSDF_CHECKED")
    os.makedirs(out_dir, exist_ok=True)
    deps = _deps()
    if not force and not _stale(lib_path, deps):
        return lib_path
    nvcc = nvcc_path()
    cuda_home = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    libdir = os.path.join(cuda_home, "lib64")

    def compile_one(src):
        obj = os.path.join(out_dir, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra_flags, "-I", INCLUDE, "-I", CSRC, "-c",
               os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for _, err in results:
            print(err)
    tmp = lib_path + f".{os.getpid()}.tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results], "-cudart", "shared",
           "-Xlinker", f"-rpath,{libdir}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib_path)
    return lib_path


def build_all(force: bool = False) -> tuple:
    """The default and the checked library, compiled side by side."""
    with ThreadPoolExecutor(max_workers=2) as ex:
        a = ex.submit(build_library, force)
        b = ex.submit(build_library, force, checked=True)
        return a.result(), b.result()


if __name__ == "__main__":
    import sys
    print(build_library(force=True, verbose="-v" in sys.argv,
                        checked="--checked" in sys.argv))
