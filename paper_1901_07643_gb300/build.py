"""Build libgivensbn.so (sm_103a) in-tree from csrc/ with nvcc, objects compiled in parallel.

Usage: python -m paper_1901_07643_gb300.build [--force] [--jobs N]
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import glob
import os
import subprocess
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "lib", "libgivensbn.so")
# checked variant: every computed index bounds-checked, synchronised per stage
OBJ_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "lib", "libgivensbn_checked.so")
# timing variant: per-role cycle counters in the workspace status block
OBJ_TIMING = os.path.join(HERE, "_build_timing")
LIB_TIMING = os.path.join(HERE, "lib", "libgivensbn_timing.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-std=c++17", "--expt-relaxed-constexpr", "-lineinfo",
                     "-Xcompiler", "-fPIC", "-I", INCLUDE]

# (scalar type, Q) pairs the dispatcher references
WALK_INSTANCES = [("float", q) for q in range(2, 10)] + [("double", q) for q in range(2, 9)]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _jobs(obj_dir=OBJ, extra=()):
    src_common = sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [os.path.join(INCLUDE, "givensbn.h")]
    jobs = []
    for name in ("r0", "roots", "api", "walk_dispatch", "noalloc", "backward", "batched", "fixup",
                 "tune", "coef", "search", "peaks", "bge", "scale"):
        src = os.path.join(CSRC, name + ".cu")
        jobs.append((os.path.join(obj_dir, name + ".o"), [src], [src] + src_common, list(extra)))
    inst = os.path.join(CSRC, "walk_inst.cu")
    for t, q in WALK_INSTANCES:
        for cov in (0, 1):
            obj = os.path.join(obj_dir, f"walk_{t}_q{q}_c{cov}.o")
            jobs.append((obj, [inst], [inst] + src_common,
                         [f"-DGBN_T={t}", f"-DGBN_Q={q}", f"-DGBN_COV={cov}"] + list(extra)))
    return jobs


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, jobs: int = 0, verbose: bool = False, checked: bool = False,
          timing: bool = False) -> str:
    if checked:
        obj_dir, lib, extra = OBJ_CHECKED, LIB_CHECKED, ["-DGBN_CHECKED"]
    elif timing:
        obj_dir, lib, extra = OBJ_TIMING, LIB_TIMING, ["-DGBN_TIMING"]
    else:
        obj_dir, lib, extra = OBJ, LIB, []
    os.makedirs(obj_dir, exist_ok=True)
    os.makedirs(os.path.dirname(lib), exist_ok=True)
    nvcc = _nvcc()
    all_jobs = _jobs(obj_dir, extra)
    todo = [j for j in all_jobs if force or _stale(j[0], j[2])]
    t0 = time.time()

    def run(job):
        obj, srcs, _, defs = job
        tmp = obj + f".tmp{os.getpid()}"
        cmd = [nvcc] + NVCC_FLAGS + defs + ["-c", srcs[0], "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {obj}:\n{r.stderr}")
        os.replace(tmp, obj)
        return obj

    if todo:
        workers = jobs or max(1, os.cpu_count() or 1)
        # largest instantiations first so the pool finishes together
        with cf.ThreadPoolExecutor(max_workers=workers) as ex:
            for obj in ex.map(run, todo):
                if verbose:
                    print(f"  built {os.path.basename(obj)} ({time.time() - t0:.0f}s)", flush=True)
    objs = [j[0] for j in all_jobs]
    if force or todo or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, lib)
    if verbose:
        print(f"{os.path.basename(lib)} ready ({time.time() - t0:.0f}s)")
    return lib


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--jobs", type=int, default=0)
    ap.add_argument("--checked", action="store_true")
    ap.add_argument("--timing", action="store_true")
    a = ap.parse_args()
    build(force=a.force, jobs=a.jobs, verbose=True, checked=a.checked, timing=a.timing)
    sys.exit(0)
