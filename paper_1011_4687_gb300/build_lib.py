"""Compile the CUDA library in-tree for sm_103a.

    python -m paper_1011_4687_gb300.build_lib [--force] [-v]

Produces paper_1011_4687_gb300/_lib/libesp_gb300.so from csrc/ with nvcc
(one -gencode: compute_103a / sm_103a) and g++ for the host-only builder.
csrc/esp_shape.cu is compiled once per launch shape listed in
csrc/esp_shapes.h (one object each); all translation units compile in
parallel; nothing else is built.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import glob
import os
import re
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libesp_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
                     "-Xcompiler", "-fPIC,-O2", "-I" + os.path.join(ROOT, "include")]
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-Wall", "-Wno-unknown-pragmas",
             "-I" + os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


SHAPE_SRC = os.path.join(CSRC, "esp_shape.cu")
SHAPE_LISTS = os.path.join(CSRC, "esp_shapes.h")


def sources():
    return sorted(p for p in glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp"))
                  if p != SHAPE_SRC)


def shape_jobs():
    """(object name, -D flags) for every launch shape listed in esp_shapes.h."""
    with open(SHAPE_LISTS) as f:
        text = f.read()
    jobs = []
    for fam in ("F32C", "F64", "BATCH"):
        m = re.search(r"#define ESP_%s_SHAPES\(X\)(.*)" % fam, text)
        if not m:
            raise RuntimeError("esp_shapes.h: no ESP_%s_SHAPES list" % fam)
        for args in re.findall(r"X\(([^)]*)\)", m.group(1)):
            v = [int(x) for x in args.split(",")]
            flags = ["-DESP_SHAPE_%s" % fam, "-DESP_NT=%d" % v[0], "-DESP_PPT=%d" % v[1]]
            if fam == "BATCH":
                flags.append("-DESP_PREC=%d" % v[2])
            jobs.append(("esp_shape_%s_%s.o" % (fam.lower(), "_".join(map(str, v))), flags))
    return jobs


def _inputs():
    return (sources() + [SHAPE_SRC] + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
            + [os.path.join(ROOT, "include", "esp.h"), os.path.abspath(__file__)])


def is_stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _inputs())


def _compile(src: str, obj: str, verbose: bool, ptxas_v: bool, defines=()) -> str:
    if src.endswith(".cu"):
        cmd = ([_nvcc()] + NVCC_FLAGS + list(defines) + (["-Xptxas", "-v"] if ptxas_v else [])
               + ["-c", src, "-o", obj])
    else:
        cmd = [os.environ.get("CXX", "g++")] + CXX_FLAGS + ["-c", src, "-o", obj]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("compile failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    return r.stderr


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False) -> str:
    if not force and not is_stale():
        return LIB
    os.makedirs(os.path.join(OUT, "obj"), exist_ok=True)
    jobs = [(s, os.path.join(OUT, "obj", os.path.basename(s) + ".o"), ()) for s in sources()]
    jobs += [(SHAPE_SRC, os.path.join(OUT, "obj", name), flags) for name, flags in shape_jobs()]
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        logs = list(ex.map(lambda j: _compile(j[0], j[1], verbose, ptxas_v, j[2]), jobs))
    objs = [j[1] for j in jobs]
    if ptxas_v:
        for j, log in zip(jobs, logs):
            if log.strip():
                print("== %s\n%s" % (os.path.basename(j[1]), log))
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ([_nvcc()] + ARCH + ["-shared", "-Xlinker", "--no-undefined", "-o", tmp] + objs
           + ["-lcudart_static", "-lrt", "-lpthread", "-ldl"])
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("-v", "--verbose", action="store_true")
    ap.add_argument("--ptxas-v", action="store_true", help="print register/smem usage per kernel")
    a = ap.parse_args(argv)
    print(build(force=a.force or a.ptxas_v, verbose=a.verbose, ptxas_v=a.ptxas_v))
    return 0


if __name__ == "__main__":
    sys.exit(main())
