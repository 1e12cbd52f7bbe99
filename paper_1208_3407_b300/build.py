"""Compile the CUDA library (csrc/*.cu) for sm_103a into libbits_b300.so,
and the random-read probe (csrc/probe.cu, a measurement aid) into
libbits_probe.so beside it.

Run as ``python -m paper_1208_3407_b300.build`` or through
``__graft_entry__.build()``.  Objects go to ``_build/`` next to this file;
``_build/ptxas.log`` keeps the register / spill / shared-memory report of
every kernel.  nvcc cross-compiles, so no GPU is needed.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libbits_b300.so")
LIB_PROBE = os.path.join(HERE, "libbits_probe.so")
PROBE_OBJS = {"probe.o"}  # measurement aid, linked into LIB_PROBE only

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-Xptxas", "-v",
         "--expt-relaxed-constexpr", f"-I{INCLUDE}"]


def _deps() -> list[str]:
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def _needs(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(p) > t for p in [src, __file__] + _deps())


def _compile(src: str) -> tuple[str, str]:
    obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
    if not _needs(obj, src):
        return obj, ""
    cmd = [NVCC, *ARCH, *FLAGS, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    with open(obj[:-2] + ".ptxas", "w") as f:
        f.write(r.stderr)
    return obj, r.stderr


def _link(out: str, objs: list[str], extra: list[str]) -> None:
    deps = objs + [x for x in extra if x.endswith(".so")]
    if os.path.exists(out) and all(os.path.getmtime(o) <= os.path.getmtime(out) for o in deps):
        return
    cmd = [NVCC, *ARCH, "-shared", "-o", out, *objs, *[x for x in extra if not x.endswith(".so")]]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link of {out} failed:\n{r.stdout}\n{r.stderr}")


def build(verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(_compile, srcs))
    with open(os.path.join(BUILD, "ptxas.log"), "w") as f:
        for p in sorted(glob.glob(os.path.join(BUILD, "*.ptxas"))):
            f.write(open(p).read())
    objs = [o for o, _ in results if os.path.basename(o) not in PROBE_OBJS]
    probe_objs = [o for o, _ in results if os.path.basename(o) in PROBE_OBJS]
    _link(LIB, objs, [])
    # The measurement probe is a library of its own that resolves the error
    # reporting helpers from libbits_b300.so next to it.
    _link(LIB_PROBE, probe_objs, [LIB, f"-L{HERE}", "-lbits_b300", "-Xlinker", "-rpath,$ORIGIN"])
    if verbose:
        print(LIB)
        print(LIB_PROBE)
    return LIB


if __name__ == "__main__":
    build(verbose=True)
    sys.exit(0)
