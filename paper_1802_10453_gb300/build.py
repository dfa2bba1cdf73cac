"""In-tree build of the CUDA libraries for sm_103a (nvcc, no cmake).

    python -m paper_1802_10453_gb300.build [--force] [--chain-profile]

produces ``libldlt_rpm.so`` (the factorisation, C ABI of include/ldlt_rpm.h)
and ``libldlt_gen.so`` (the GPU input generator) next to this file.  Sources
compile in parallel; a library is rebuilt only when a source is newer.
--chain-profile rebuilds everything with LDLT_CHAIN_PROFILE defined: the
pivot chain then also records SM-cycle counters per leader phase and per
barrier (ldlt_rpm_profile_read out[8..15], out[26..31]); a later plain build
must be forced to drop them.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(ROOT, "_build")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include")]

LIBS = {
    "libldlt_rpm.so": ["panel.cu", "kernels_misc.cu", "syrdk_fp64.cu", "syrdk_tc.cu", "ldlt_rpm.cu",
                       "noalloc.cu", "batched.cu", "strict_char2.cu",
                       "solve.cu", "trss.cu", "given.cu"],
    "libldlt_gen.so": ["gen_kernels.cu"],
}
HEADERS = ["field.cuh", "ldlt_internal.cuh"]


def _newest(paths):
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False, chain_profile: bool = False) -> dict:
    flags = FLAGS + (["-DLDLT_CHAIN_PROFILE"] if chain_profile else [])
    force = force or chain_profile
    os.makedirs(BUILD, exist_ok=True)
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "ldlt_rpm.h")]
    out = {}
    jobs = []
    plan = []
    for lib, srcs in LIBS.items():
        target = os.path.join(HERE, lib)
        paths = [os.path.join(CSRC, s) for s in srcs]
        stale = force or not os.path.exists(target) or os.path.getmtime(target) < _newest(paths + hdrs)
        objs = []
        for s in paths:
            o = os.path.join(BUILD, os.path.basename(s) + ".o")
            objs.append(o)
            if stale and (force or not os.path.exists(o) or os.path.getmtime(o) < _newest([s] + hdrs)):
                cmd = [NVCC] + ARCH + flags + ["-c", s, "-o", o]
                jobs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        plan.append((lib, target, objs, stale))
        out[lib] = target
    for cmd, pr in jobs:
        txt, _ = pr.communicate()
        if pr.returncode != 0:
            sys.stderr.write(txt.decode(errors="replace"))
            raise RuntimeError("nvcc failed: " + " ".join(cmd))
        if verbose and txt:
            sys.stderr.write(txt.decode(errors="replace"))
    for lib, target, objs, stale in plan:
        if stale:
            tmp = target + ".tmp%d" % os.getpid()
            cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, target)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, chain_profile="--chain-profile" in sys.argv))
