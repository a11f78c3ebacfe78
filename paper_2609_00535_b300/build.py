"""Build the package's CUDA libraries in-tree with nvcc for sm_103a (B300).

Each source is compiled to an object in parallel, then linked into the shared
library next to this file (the binding loads it from here).
"""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2"]
OBJDIR = os.path.join(ROOT, "_build")

TARGETS = {
    "libsemlbm.so": ["csrc/sem_lbm.cu", "csrc/batch.cu"],
    "libsemlbm_peak.so": ["csrc/fp64_peak.cu"],
}


def _deps():
    out = []
    for d in (os.path.join(HERE, "csrc"), os.path.join(ROOT, "include")):
        out += [os.path.join(d, f) for f in os.listdir(d)]
    return out


def _stale(out):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(p) > t for p in _deps())


def _run(cmd, verbose):
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.run(cmd, check=True)


def build(force=False, verbose=True):
    os.makedirs(OBJDIR, exist_ok=True)
    inc = ["-I", os.path.join(ROOT, "include")]
    jobs = []
    for name, srcs in TARGETS.items():
        out = os.path.join(HERE, name)
        if force or _stale(out):
            jobs.append((out, [os.path.join(HERE, s) for s in srcs]))
    compile_cmds = []
    for out, srcs in jobs:
        for src in srcs:
            obj = os.path.join(OBJDIR, os.path.basename(src) + ".o")
            compile_cmds.append([NVCC] + ARCH + FLAGS + inc + ["-c", "-o", obj, src])
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(compile_cmds), os.cpu_count() or 1))) as ex:
        for f in [ex.submit(_run, c, verbose) for c in compile_cmds]:
            f.result()
    for out, srcs in jobs:
        objs = [os.path.join(OBJDIR, os.path.basename(s) + ".o") for s in srcs]
        _run([NVCC] + ARCH + ["-shared", "-o", out + ".tmp"] + objs, verbose)
        os.replace(out + ".tmp", out)


if __name__ == "__main__":
    build(force="--force" in sys.argv)
