"""Builds libdirac.so (the CUDA library behind include/dirac.h) in place with nvcc for
sm_103a. Translation units compile in parallel; the result is linked with the static
CUDA runtime so the library has no runtime dependency beyond the driver."""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
# DIRAC_BUILD_TAG=<tag> builds libdirac_<tag>.so (objects in _build_<tag>) beside the
# default library, e.g. a debug build with DIRAC_NVCC_EXTRA="-DDIRAC_DEBUG=1".
_TAG = os.environ.get("DIRAC_BUILD_TAG", "")
BUILD = os.path.join(HERE, "_build" + (f"_{_TAG}" if _TAG else ""))
LIB = os.path.join(HERE, "libdirac" + (f"_{_TAG}" if _TAG else "") + ".so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _deps():
    return (glob.glob(os.path.join(CSRC, "*")) +
            [os.path.join(HERE, "..", "include", "dirac.h"), __file__])


def _extra_flags():
    """Extra nvcc flags from DIRAC_NVCC_EXTRA (e.g. "-DDGB_PACKED_F32X2=0"), split on
    whitespace; a change of them forces a rebuild."""
    return os.environ.get("DIRAC_NVCC_EXTRA", "").split()


def build(force: bool = False, verbose: bool = False) -> str:
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    newest = max(os.path.getmtime(p) for p in _deps())
    extra = _extra_flags()
    stamp = LIB + ".flags"
    old_extra = open(stamp).read() if os.path.exists(stamp) else ""
    if (not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest
            and old_extra == " ".join(extra)):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    procs = []
    objs = []
    for src in sources:
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((src, out.decode(errors="replace")))
    if failed:
        msg = "\n".join(f"{s}:\n{o}" for s, o in failed)
        raise RuntimeError(f"nvcc failed:\n{msg}")
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], check=True)
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(" ".join(extra))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
