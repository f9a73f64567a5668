"""Builds libmbinv.so in-tree with nvcc for sm_103a (no CMake).

Every translation unit is compiled in parallel, then linked into
``paper_1612_00001_gb300/_build/libmbinv.so`` (the product) and the test
hooks of ``csrc/testhooks`` into ``_build/libmbinv_test.so``, which links
against the product library and is loaded only by the tests and the bench.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmbinv.so")
TEST_SRC = os.path.join(CSRC, "testhooks")
TEST_LIB = os.path.join(BUILD, "libmbinv_test.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmbinv")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def test_sources():
    return sorted(os.path.join(TEST_SRC, f) for f in os.listdir(TEST_SRC) if f.endswith((".cu", ".cpp")))


def _stale() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(TEST_LIB):
        return True
    t = min(os.path.getmtime(LIB), os.path.getmtime(TEST_LIB))
    deps = ([os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(TEST_SRC, f) for f in os.listdir(TEST_SRC)]
            + [os.path.join(HERE, "..", "include", "mbinv.h"), os.path.abspath(__file__)])
    return any(os.path.getmtime(d) > t for d in deps if os.path.isfile(d))


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    common = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                     "-I", os.path.join(HERE, "..", "include"), "-I", CSRC]

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        cmd = [nvcc] + common + ["-c", src, "-o", obj]
        if src.endswith(".cpp"):
            cmd = [nvcc] + common + ["-x", "c++", "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr, file=sys.stderr)
        return obj

    srcs = sources()
    tsrcs = test_sources()
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs) + len(tsrcs))) as ex:
        objs = list(ex.map(compile_one, srcs + tsrcs))
    objs, tobjs = objs[:len(srcs)], objs[len(srcs):]

    def link(out, cmd_tail):
        tmp = out + f".{os.getpid()}.tmp"
        r = subprocess.run([nvcc] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + cmd_tail,
                           capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link of {os.path.basename(out)} failed:\n{r.stderr}")
        os.replace(tmp, out)

    link(LIB, objs)
    # the test hooks call into the product library, found next to them
    link(TEST_LIB, tobjs + ["-L", BUILD, "-lmbinv", "-Xlinker", "-rpath", "-Xlinker", "$ORIGIN"])
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
