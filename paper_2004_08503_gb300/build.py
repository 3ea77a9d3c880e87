"""Build libsidp.so in-tree for sm_103a (nvcc only; translation units compiled in parallel).

    python -m paper_2004_08503_gb300.build [--force] [-j N]
"""
import argparse
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libsidp.so")
NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-ftz=true", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include"),
         "-diag-suppress", "177"]
SOURCES = ["sidp_api.cu", "sidp_batch.cu", "sidp_tables.cpp", "sidp_geometry.cpp", "sidp_noalloc.cu", "sidp_peaks.cu",
           "inst_burgers_f64.cu", "inst_burgers_f32.cu", "inst_advection_f64.cu", "inst_advection_f32.cu",
           "inst_advection_var_f64.cu", "inst_advection_var_f32.cu",
           "inst_euler_f64_a.cu", "inst_euler_f64_b.cu", "inst_euler_f64_c.cu",
           "inst_euler_f32_a.cu", "inst_euler_f32_b.cu", "inst_euler_f32_c.cu",
           "inst_batch_all_f32.cu", "inst_batch_all_f64.cu"]


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs.append(os.path.join(ROOT, "include", "sidp.h"))
    return hs


def _stale(obj, src, hdr_mtime):
    return not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(src), hdr_mtime)


def build(force=False, jobs=None, verbose=False):
    os.makedirs(BUILD, exist_ok=True)
    hdr_mtime = max(os.path.getmtime(h) for h in _headers())
    todo = []
    objs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD, s + ".o")
        objs.append(obj)
        if force or _stale(obj, src, hdr_mtime):
            lang = ["-x", "cu"] if s.endswith(".cu") else ["-x", "c++"]
            todo.append([NVCC] + ARCH + FLAGS + lang + ["-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0 or verbose:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.returncode

    if todo:
        with ThreadPoolExecutor(max_workers=jobs or min(len(todo), os.cpu_count() or 4)) as ex:
            codes = list(ex.map(run, todo))
        if any(codes):
            raise RuntimeError("libsidp compilation failed")
    if force or todo or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        cmd = [NVCC] + ARCH + ["-shared", "-o", LIB] + objs
        if run(cmd):
            raise RuntimeError("libsidp link failed")
    return LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("-j", type=int, default=None)
    ap.add_argument("-v", action="store_true")
    a = ap.parse_args()
    print(build(a.force, a.j, a.v))
