"""Builds ``libsts.so`` in-tree from ``csrc/*.cu`` with nvcc for sm_103a.

Each translation unit compiles in parallel; ``sts_tree.cu`` (every FP64 decision of the
tree: faces, child digits, MAC) additionally gets ``--fmad=false``.  Host code is compiled
with ``-ffp-contract=off`` so that the icosahedron and the proxy tables are plain IEEE
double arithmetic on x86 and Arm alike.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsts.so")

SOURCES = ["sts_api.cu", "sts_tables.cu", "sts_scan.cu", "sts_tree.cu", "sts_upward.cu",
           "sts_eval.cu", "sts_down.cu", "sts_rk4.cu", "sts_amr.cu", "sts_tc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC,-ffp-contract=off",
              "-Xptxas", "-v"]
PER_FILE = {"sts_tree.cu": ["--fmad=false"], "sts_amr.cu": ["--fmad=false"]}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _deps():
    out = [os.path.join(CSRC, s) for s in SOURCES]
    out += [os.path.join(CSRC, "sts_internal.cuh"), os.path.join(INCLUDE, "sts.h"), __file__]
    return out


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles every translation unit and links ``libsts.so``; returns its path."""
    if not force and not needs_build():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        log = os.path.join(BUILD, src.replace(".cu", ".log"))
        objs.append(obj)
        cmd = [cc, *NVCC_FLAGS, *PER_FILE.get(src, []), "-I", INCLUDE, "-c",
               os.path.join(CSRC, src), "-o", obj]
        procs.append((src, log, subprocess.Popen(cmd, stdout=open(log, "w"), stderr=subprocess.STDOUT)))
    failed = []
    for src, log, p in procs:
        if p.wait() != 0:
            failed.append((src, log))
    if failed:
        msg = []
        for src, log in failed:
            with open(log) as f:
                msg.append(f"--- {src}\n" + f.read()[-4000:])
        raise RuntimeError("nvcc failed:\n" + "\n".join(msg))
    if verbose:
        for src, log, _ in procs:
            with open(log) as f:
                sys.stdout.write(f"--- {src}\n" + f.read())
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([cc, "-shared", *ARCH, "-o", tmp, *objs])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
