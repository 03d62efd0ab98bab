"""Builds libsquares.so (the C-ABI library) for sm_103a with nvcc.

Each translation unit is compiled in parallel into ``_build/`` and linked
in-tree as ``paper_2004_06278_gb300/libsquares.so``. The CUDA runtime is
linked statically (nvcc's default), so the library needs only the driver.
"""
from __future__ import annotations

import hashlib
import os
import re
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libsquares.so")

SOURCES = ["api.cpp", "keys.cpp", "kernels_plain.cu", "kernels_batch.cu", "kernels_fused.cu",
           "kernels_misc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# The device code: a tuned launch table is valid only for the library built
# from these sources (sq_build_id, sq_autotune_save / _load).
KERNEL_SOURCES = [os.path.join(CSRC, f) for f in ("kernels_plain.cu", "kernels_batch.cu",
                                                  "kernels_fused.cu", "kernels_misc.cu",
                                                  "stores.cuh", "internal.h")] + [
    os.path.join(INCLUDE, "squares_device.cuh")]


def code_only(text: str) -> str:
    """C/C++/CUDA source without comments and whitespace: what the compiler
    sees, so that edits to comments do not change an identifier."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return re.sub(r"\s+", "", text)


def code_hash(paths) -> str:
    """First 16 hex digits of the SHA-256 of the sources' code."""
    h = hashlib.sha256()
    for p in paths:
        with open(p, encoding="utf-8") as f:
            h.update(code_only(f.read()).encode())
    return h.hexdigest()[:16]


def build_id() -> str:
    """Identifier of the kernel code (see KERNEL_SOURCES)."""
    return code_hash(KERNEL_SOURCES)


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsquares.so")


def _flags(verbose: bool) -> list[str]:
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-I", INCLUDE,
                "-I", CSRC]
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def _id_stamp(obj: str) -> str:
    return obj + ".id"


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    deps = [src, os.path.join(CSRC, "stores.cuh"), os.path.join(CSRC, "internal.h"),
            os.path.join(INCLUDE, "squares.h"), os.path.join(INCLUDE, "squares_device.cuh"), __file__]
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    bid = build_id()
    jobs = []
    objs = []
    stamps = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD, s + ".o")
        objs.append(obj)
        extra = []
        stale = force or _stale(obj, src)
        if s == "api.cpp":
            # the C ABI reports the kernel code it was built with
            extra = [f"-DSQ_BUILD_ID=\"{bid}\""]
            stamp = _id_stamp(obj)
            old = open(stamp).read().strip() if os.path.exists(stamp) else None
            stale = stale or old != bid
            if stale:
                stamps.append((stamp, bid))
        if stale:
            jobs.append([cc, *_flags(verbose), *extra, "-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    failed = []
    with ThreadPoolExecutor(max_workers=len(jobs) or 1) as ex:
        for cmd, r in ex.map(run, jobs):
            if verbose or r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode != 0:
                failed.append(cmd[-3])
    if failed:
        raise RuntimeError(f"nvcc failed for {failed}")
    for stamp, value in stamps:
        with open(stamp, "w") as f:
            f.write(value + "\n")
    if jobs or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
