"""Build the b3phys CUDA library in-tree (sm_103a) with nvcc."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = [os.path.join(HERE, "csrc", f) for f in ("b3p_step.cu", "b3p_host.cpp", "b3p_server.cpp")]
DEPS = SRC + [os.path.join(HERE, "csrc", "b3p_internal.h"),
              os.path.join(os.path.dirname(HERE), "include", "b3phys.h")]
LIB = os.path.join(HERE, "libb3phys.so")
TRACE_LIB = os.path.join(HERE, "libb3phys_trace.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_cmd(out: str, extra=()):
    return (["nvcc", "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-shared",
             "-cudart", "shared", "-Xlinker", "-rpath,/usr/local/cuda/lib64", "-Xptxas", "-v", *extra, "-o", out, *SRC])


def build(force: bool = False, verbose: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and all(os.path.getmtime(LIB) >= os.path.getmtime(d) for d in DEPS)):
        return LIB
    tmp = LIB + ".tmp"
    r = subprocess.run(nvcc_cmd(tmp), capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc failed building libb3phys.so")
    if verbose:
        sys.stderr.write(r.stderr)
    os.replace(tmp, LIB)
    return LIB


CHECKED_LIB = os.path.join(HERE, "libb3phys_checked.so")
NOFMA_LIB = os.path.join(HERE, "libb3phys_nofma.so")


def _variant(out: str, flags: tuple, force: bool) -> str:
    if (not force and os.path.exists(out)
            and all(os.path.getmtime(out) >= os.path.getmtime(d) for d in DEPS)):
        return out
    r = subprocess.run(nvcc_cmd(out + ".tmp", extra=flags), capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError(f"nvcc failed building {os.path.basename(out)}")
    os.replace(out + ".tmp", out)
    return out


def build_checked(force: bool = False) -> str:
    """The checked variant (index checks on the per-world accessors and update lists,
    b3p_check_read); used by the tests in place of a memory checker, not by the product
    path."""
    return _variant(CHECKED_LIB, ("-DB3P_CHECKED",), force)


def build_trace(force: bool = False) -> str:
    """The tracing variant (per-stage clock64 totals, b3p_trace_read); not used by the
    product path."""
    return _variant(TRACE_LIB, ("-DB3P_TRACE",), force)


def build_nofma(force: bool = False) -> str:
    """The same sources without fused multiply-add contraction (-fmad=false); the tests
    use it to show that two code paths run the same arithmetic, which the default build
    may round differently where the compiler fuses a product into a sum in one kernel and
    not in another. Not used by the product path."""
    return _variant(NOFMA_LIB, ("-fmad=false",), force)


if __name__ == "__main__":
    build(force=True, verbose=True)
    print(LIB)
