"""Build librqa_b300.so in-tree: CUDA sources for sm_103a with nvcc, host
sources with g++ (-ffp-contract=off, so the host measures never fuse a
multiply-add), linked into one shared library next to this file.

    python -m paper_2402_16853_b300.build [--force] [--debug]
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "librqa_b300.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _sources():
    cu = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    cpp = sorted(glob.glob(os.path.join(CSRC, "*.cpp")))
    hdr = sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
                 + glob.glob(os.path.join(INCLUDE, "*.h")))
    return cu, cpp, hdr


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, debug: bool = False, verbose: bool = False) -> str:
    cu, cpp, hdr = _sources()
    if not force and not _stale(LIB, cu + cpp + hdr + [__file__]):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    opt = ["-O0", "-g"] if debug else ["-O3"]
    jobs = []
    for src in cu:
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        if force or _stale(obj, [src] + hdr + [__file__]):
            jobs.append([nvcc, ARCH, "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
                         "-Xcompiler", "-ffp-contract=off", f"-I{INCLUDE}", "-c", src, "-o", obj]
                        + opt)
    for src in cpp:
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        if force or _stale(obj, [src] + hdr + [__file__]):
            jobs.append(["g++", "-std=c++17", "-fPIC", "-ffp-contract=off", "-fno-fast-math",
                         "-Wall", "-Wextra", f"-I{INCLUDE}", "-I/usr/local/cuda/include", "-c",
                         src, "-o", obj] + (["-O0", "-g"] if debug else ["-O2"]))
    with cf.ThreadPoolExecutor(max_workers=max(1, os.cpu_count() or 1)) as ex:
        futs = [ex.submit(subprocess.run, j, capture_output=True, text=True) for j in jobs]
        errs = []
        for j, f in zip(jobs, futs):
            r = f.result()
            if verbose or r.returncode:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode:
                errs.append(" ".join(j))
        if errs:
            raise RuntimeError("compilation failed:\n" + "\n".join(errs))
    objs = [os.path.join(BUILD, os.path.basename(s) + ".o") for s in cu + cpp]
    tmp = LIB + f".{os.getpid()}.tmp"
    link = [nvcc, ARCH, "-shared", "-o", tmp] + objs + ["-lcudart", "-lpthread"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode:
        raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    return LIB


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--debug", action="store_true")
    ap.add_argument("-v", "--verbose", action="store_true")
    a = ap.parse_args()
    print(build(force=a.force, debug=a.debug, verbose=a.verbose))


if __name__ == "__main__":
    main()
