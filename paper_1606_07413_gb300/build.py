"""Build libqcs.so in-tree with nvcc for sm_103a (GB300).

Sources are compiled in parallel, one process per translation unit, then
linked into ``paper_1606_07413_gb300/_build/libqcs.so`` with only the ``qcs_*``
symbols of include/qcs.h exported.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libqcs.so")

SOURCES = ["qcs_walk.cu", "qcs_api.cpp", "qcs_exact.cpp", "qcs_noalloc.cu", "qcs_batch.cpp"]
PEAK_SRC = "qcs_peak.cu"
PEAK_LIB = os.path.join(BUILD, "libqcs_peak.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libqcs")


def _inputs():
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += [os.path.join(CSRC, "qcs_internal.h"), os.path.join(INCLUDE, "qcs.h"), __file__,
              os.path.join(CSRC, PEAK_SRC), os.path.join(INCLUDE, "qcs_peak.h")]
    return files


def up_to_date() -> bool:
    if not (os.path.exists(LIB) and os.path.exists(PEAK_LIB)):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(PEAK_LIB))
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    common = ["-O3", "-std=c++17", "-I", INCLUDE, "-I", CSRC, "-Xcompiler", "-fPIC,-fvisibility=hidden",
              *ARCH, "-lineinfo", *extra_flags]
    procs, objs = [], []
    peak_tmp = PEAK_LIB + f".{os.getpid()}.tmp"
    peak_cmd = [cc, *common, "-shared", "-o", peak_tmp, os.path.join(CSRC, PEAK_SRC),
                "-Xlinker", "--version-script=" + os.path.join(BUILD, "peak.map")]
    with open(os.path.join(BUILD, "peak.map"), "w") as f:
        f.write("{ global: qcs_peak_*; local: *; };\n")
    procs.append((peak_cmd, subprocess.Popen(peak_cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for s in SOURCES:
        obj = os.path.join(BUILD, os.path.basename(s) + ".o")
        objs.append(obj)
        cmd = [cc, *common, "-c", os.path.join(CSRC, s), "-o", obj]
        if s.endswith(".cu"):
            cmd += ["-Xptxas", "-v"] if verbose else []
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    tmp = LIB + f".{os.getpid()}.tmp"
    try:
        failed = []
        for cmd, p in procs:
            out, _ = p.communicate()
            if verbose or p.returncode:
                sys.stderr.write(out.decode(errors="replace"))
            if p.returncode:
                failed.append(" ".join(cmd))
        if failed:
            raise RuntimeError("libqcs build failed:\n" + "\n".join(failed))
        vers = os.path.join(BUILD, "exports.map")
        with open(vers, "w") as f:
            f.write("{ global: qcs_*; local: *; };\n")
        link = [cc, "-shared", *ARCH, "-o", tmp, *objs, "-Xlinker", f"--version-script={vers}", "-lpthread"]
        subprocess.check_call(link)
        os.replace(tmp, LIB)
        os.replace(peak_tmp, PEAK_LIB)
    finally:
        # a failed build leaves no half-written library behind
        for f in (tmp, peak_tmp):
            if os.path.exists(f):
                os.remove(f)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
