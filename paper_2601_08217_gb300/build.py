"""Build libttchan.so in-tree with nvcc for sm_103a (GB300).

Each translation unit compiles in parallel; the result lands in
``paper_2601_08217_gb300/_build/libttchan.so`` (git-ignored), beside the bounds-checked
``libttchan_checked.so`` (kernels compiled with TT_CHECKED=1).  Nothing here needs
a GPU: nvcc cross-compiles.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libttchan.so")
LIB_CHECKED = os.path.join(OUT, "libttchan_checked.so")  # bounds-checked build (TT_CHECKED=1)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libttchan.so")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _digest() -> str:
    h = hashlib.sha256()
    for f in sorted(os.listdir(CSRC)) + ["../build.py"]:
        p = os.path.join(CSRC, f)
        if os.path.isfile(p):
            h.update(f.encode())
            h.update(open(p, "rb").read())
    h.update(open(os.path.join(INCLUDE, "tt_chan.h"), "rb").read())
    h.update(os.uname().machine.encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    """Build libttchan.so and its bounds-checked twin libttchan_checked.so (the .cu translation units
    compiled again with TT_CHECKED=1, linked with the same host objects); returns the first's path."""
    os.makedirs(os.path.join(OUT, "checked"), exist_ok=True)
    stamp = os.path.join(OUT, "stamp")
    dig = _digest()
    if (not force and os.path.exists(LIB) and os.path.exists(LIB_CHECKED) and os.path.exists(stamp)
            and open(stamp).read() == dig):
        return LIB
    nvcc = _nvcc()

    def compile_one(job):
        src, checked = job
        obj = os.path.join(OUT, "checked" if checked else "", os.path.basename(src) + ".o")
        cmd = [nvcc] + ARCH + COMMON + (["-DTT_CHECKED=1"] if checked else []) + ["-c", src, "-o", obj]
        if src.endswith(".cpp"):
            cmd = [nvcc] + COMMON + ["-x", "c++", "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}{' (checked)' if checked else ''}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    srcs = sources()
    # the kernels of both libraries first (the longest jobs), host code once
    jobs = [(s_, False) for s_ in srcs if s_.endswith(".cu")] + [(s_, True) for s_ in srcs if s_.endswith(".cu")]
    jobs += [(s_, False) for s_ in srcs if s_.endswith(".cpp")]
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        objs = dict(zip(jobs, ex.map(compile_one, jobs)))
    host = [objs[(s_, False)] for s_ in srcs if s_.endswith(".cpp")]
    cudalib = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "lib64")
    for lib, checked in ((LIB, False), (LIB_CHECKED, True)):
        kern = [objs[(s_, checked)] for s_ in srcs if s_.endswith(".cu")]
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-Xlinker", "-rpath", "-Xlinker", cudalib,
                               "-o", tmp] + kern + host + ["-lpthread", "-ldl"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    open(stamp, "w").write(dig)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
