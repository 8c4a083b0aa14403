"""Build the sm_103a shared library in-tree (nvcc, no torch extension machinery).

``build()`` compiles the ``csrc/*.cu`` translation units into ``libzk.so`` next to this file.
The library exports the C ABI of ``include/zk.h`` and links the CUDA runtime
statically, so it loads with nothing but the driver.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libzk.so")
SOURCES = [os.path.join(HERE, "csrc", f) for f in (
    "zk_api.cu", "zk_static.cu", "zk_net.cu", "zk_launch_common.cu",
    "zk_launch_row_f32.cu", "zk_launch_row_f64.cu", "zk_launch_col_f32.cu", "zk_launch_col_f64.cu")]
DEPS = sorted(os.path.join(HERE, "csrc", f) for f in os.listdir(os.path.join(HERE, "csrc"))
              if f.endswith((".cu", ".cuh", ".h"))) + [os.path.join(ROOT, "include", "zk.h")]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in DEPS if os.path.exists(d))


def build(force: bool = False, verbose: bool = False, extra=None) -> str:
    """Compile each translation unit in parallel, then link libzk.so."""
    if not force and up_to_date():
        return LIB
    flags = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
    if verbose:
        flags.append("-Xptxas=-v")
    if extra:
        flags += list(extra)
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(HERE, os.path.basename(src) + ".o")
        objs.append(obj)
        procs.append((src, subprocess.Popen([nvcc(), *flags, "-c", "-o", obj, src], stdout=subprocess.PIPE,
                                            stderr=subprocess.STDOUT, text=True)))
    failed = False
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            sys.stderr.write(out)
        failed |= p.returncode != 0
    if failed:
        raise RuntimeError("nvcc failed")
    r = subprocess.run([nvcc(), *ARCH, "-shared", "-o", LIB + ".tmp", *objs], capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc link failed")
    for o in objs:
        os.remove(o)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
