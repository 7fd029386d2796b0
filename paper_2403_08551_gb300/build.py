"""Builds libgi.so (the CUDA kernels and the C ABI) in-tree for sm_103a.

``python -m paper_2403_08551_gb300.build`` or ``build()``: every .cu file in
csrc/ is compiled by nvcc in parallel (one -gencode, arch sm_103a), then
linked into ``_build/libgi.so`` with the CUDA runtime linked statically.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libgi.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-fvisibility=hidden", "-I", INCLUDE]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs.append(os.path.join(INCLUDE, "gi.h"))
    return hs


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


# Variants: "release" (the product, _build/libgi.so) and "check"
# (_build_check/libgi.so, compiled with -DGI_CHECK_BOUNDS: extra index
# checks in the kernels that raise the bounds error bit and skip the access).
VARIANTS = {"release": (OUT, []), "check": (os.path.join(HERE, "_build_check"), ["-DGI_CHECK_BOUNDS"])}


def library_path(variant: str = "release") -> str:
    return os.path.join(VARIANTS[variant][0], "libgi.so")


def build(force: bool = False, verbose: bool = False, extra_flags=None, variant: str = "release") -> str:
    out_dir, vflags = VARIANTS[variant]
    LIB = os.path.join(out_dir, "libgi.so")
    OUT = out_dir
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    flags = NVCC_FLAGS + vflags + list(extra_flags or [])
    srcs = sources()
    headers = _deps()
    objs = []
    jobs = []
    for src in srcs:
        obj = os.path.join(OUT, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + headers + [__file__]):
            jobs.append((src, obj))

    def compile_one(job):
        src, obj = job
        cmd = [nvcc] + ARCH + flags + ["-c", src, "-o", obj + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stderr}")
        os.replace(obj + ".tmp", obj)
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            list(ex.map(compile_one, jobs))
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "static"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stderr)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, variant="check" if "--check" in sys.argv else "release"))
