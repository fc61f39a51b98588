"""Build the CUDA libraries in-tree with nvcc for sm_103a (GB300):

    liblbm.so  the lattice Boltzmann solver (include/lbm.h)
    libfno.so  the kernels of the learned warm start (include/fno.h)
    libfnonet.so  the fused tensor-core kernels of that network (include/fno_net.h)

    python -m paper_1409_5929_gb300.build [--force] [-v]
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(ROOT, "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

TARGETS = {
    "liblbm.so": ([os.path.join(CSRC, "lbm.cu")],
                  [os.path.join(CSRC, "lbm_physics.cuh"), os.path.join(INC, "lbm.h")]),
    "libfno.so": ([os.path.join(CSRC, "fno.cu")], [os.path.join(INC, "fno.h")]),
    "libfnonet.so": ([os.path.join(CSRC, "fno_net.cu")], [os.path.join(CSRC, "tc.cuh"), os.path.join(INC, "fno_net.h")]),
}
LIB = os.path.join(HERE, "liblbm.so")
FNO_LIB = os.path.join(HERE, "libfno.so")


def nvcc() -> str:
    env = os.environ.get("NVCC")
    if env:
        return env
    return "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc"


def _stale(out: str, deps) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def _build_one(name: str, force: bool, verbose: bool) -> str:
    sources, headers = TARGETS[name]
    out = os.path.join(HERE, name)
    if not force and not _stale(out, sources + headers):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC", "-I", INC,
           "-o", tmp, *sources]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False, verbose: bool = False) -> str:
    with ThreadPoolExecutor(max_workers=len(TARGETS)) as ex:
        list(ex.map(lambda n: _build_one(n, force, verbose), TARGETS))
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print("\n".join(os.path.join(HERE, n) for n in TARGETS))
