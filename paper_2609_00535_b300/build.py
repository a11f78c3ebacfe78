"""Build libsemlbm.so in-tree with nvcc for sm_103a (B300)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-shared"]

TARGETS = {
    "libsemlbm.so": ["csrc/sem_lbm.cu"],
    "libsemlbm_peak.so": ["csrc/fp64_peak.cu"],
}


def _stale(out, srcs):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    deps = list(srcs)
    for d in (os.path.join(HERE, "csrc"), os.path.join(ROOT, "include")):
        for f in os.listdir(d):
            deps.append(os.path.join(d, f))
    return any(os.path.getmtime(p) > t for p in deps)


def build(force=False, verbose=True):
    for name, srcs in TARGETS.items():
        out = os.path.join(HERE, name)
        srcs = [os.path.join(HERE, s) for s in srcs]
        if not force and not _stale(out, srcs):
            continue
        cmd = [NVCC] + ARCH + FLAGS + ["-I", os.path.join(ROOT, "include"), "-o", out + ".tmp"] + srcs
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.run(cmd, check=True)
        os.replace(out + ".tmp", out)


if __name__ == "__main__":
    build(force="--force" in sys.argv)
