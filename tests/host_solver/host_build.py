"""Host build of the library's solver headers (test infrastructure).

``csrc/common.cuh`` and ``csrc/forward.cuh`` are copied with their device qualifiers dropped and
the few device intrinsics replaced by host arithmetic: the hardware reciprocal approximation by
an IEEE division, the fast exp/log by expf/logf, popc by the compiler builtin; products are
contracted into fused multiply-adds as nvcc does. The result models the device's FP32 epoch
loop closely enough to check its logic (root iteration, image selection, the MIXED triggers) on
a CPU; on the 4096 x 2000 sweep it reproduced the device's re-solve flags and failing epochs.
"""
from __future__ import annotations

import os
import platform
import re
import shutil
import subprocess

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
CSRC = os.path.join(ROOT, "paper_1208_4830_gb300", "csrc")
HERE = os.path.dirname(os.path.abspath(__file__))


def _host(src: str) -> str:
    src = src.replace(
        "#include <cuda_runtime.h>",
        "#include <cmath>\n#include <algorithm>\nusing std::isfinite; using std::fmin; using std::fmax; using std::fabs;",
    )
    src = src.replace("__device__ __forceinline__", "static inline").replace("__device__ __noinline__", "static")
    src = re.sub(r'asm\("rcp\.approx\.ftz\.f32 %0, %1;" : "=f"\(r\) : "f"\(x\)\);', "r = 1.0f / x;", src)
    src = re.sub(r'asm\("rcp\.approx\.ftz\.f64 %0, %1;" : "=d"\(r\) : "d"\(x\)\);', "r = 1.0 / x;", src)
    src = src.replace("rsqrtf(x)", "(1.0f / sqrtf(x))").replace("return rsqrt(x);", "return 1.0 / sqrt(x);")
    src = src.replace("__expf", "expf").replace("__logf", "logf").replace("__popc(", "__builtin_popcount(")
    src = src.replace("__umul64hi(", "umul64hi_host(")
    return src


def build(workdir: str) -> str:
    """Compile the host loop in ``workdir``; returns the executable's path."""
    gxx = shutil.which("g++")
    if not gxx:
        raise RuntimeError("g++ not found")
    common = _host(open(os.path.join(CSRC, "common.cuh")).read())
    common = common.replace(
        "namespace sblm {",
        "namespace sblm {\nstatic inline uint64_t umul64hi_host(uint64_t a, uint64_t b) "
        "{ return (uint64_t)(((unsigned __int128)a * b) >> 64); }",
        1,
    )
    open(os.path.join(workdir, "common.cuh"), "w").write(common)
    open(os.path.join(workdir, "forward.cuh"), "w").write(_host(open(os.path.join(CSRC, "forward.cuh")).read()))
    exe = os.path.join(workdir, "host_loop")
    flags = ["-O2", "-std=c++17", "-ffp-contract=fast"]
    if platform.machine() in ("x86_64", "AMD64"):
        flags.append("-mfma")  # fused multiply-adds, as on the GPU (native on aarch64)
    subprocess.run([gxx, *flags, "-I", workdir, os.path.join(HERE, "host_loop.cpp"), "-o", exe], check=True)
    return exe


def build_count(workdir: str) -> str:
    """Compile the operation-counting loop (count_loop.cpp) in ``workdir`` (after build())."""
    gxx = shutil.which("g++")
    exe = os.path.join(workdir, "count_loop")
    shutil.copy(os.path.join(HERE, "count_types.h"), os.path.join(workdir, "count_types.h"))
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", workdir, os.path.join(HERE, "count_loop.cpp"), "-o", exe],
                   check=True)
    return exe


def aberth_order(workdir: str):
    """Build and run aberth_order.cpp in ``workdir`` (after build()), with contraction off so that
    the two formulations round identically; returns (cases, mismatches, capped, masked)."""
    gxx = shutil.which("g++")
    exe = os.path.join(workdir, "aberth_order")
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", workdir,
                    os.path.join(HERE, "aberth_order.cpp"), "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    return tuple(int(x) for x in out)


def count(exe: str, theta, t, flux, sigma, seg: int, workdir: str, fp64: bool = False):
    """(epochs, FP32 operations, FP64 operations, epochs re-solved in FP64) of the MIXED epoch
    loop (or, with ``fp64``, the FP64 mode's loop) over every (row, epoch); runs of ``seg`` epochs
    start cold."""
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    n, m = theta.shape[0], np.asarray(t).size
    src = os.path.join(workdir, "count_in.bin")
    with open(src, "wb") as f:
        np.array([n, m, seg], dtype=np.int32).tofile(f)
        for a in (t, flux, 1.0 / np.asarray(sigma, dtype=np.float64)):
            np.ascontiguousarray(a, dtype=np.float64).tofile(f)
        theta.tofile(f)
    args = [exe, "--fp64", src] if fp64 else [exe, src]
    out = subprocess.run(args, check=True, capture_output=True, text=True).stdout.split()
    return tuple(int(x) for x in out)


def run(exe: str, theta, t, seg: int, workdir: str):
    """(A32, flags, A64) of every (row, epoch); runs of ``seg`` epochs start cold."""
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    n, m = theta.shape[0], t.size
    src, dst = os.path.join(workdir, "in.bin"), os.path.join(workdir, "out.bin")
    with open(src, "wb") as f:
        np.array([n, m, seg], dtype=np.int32).tofile(f)
        t.tofile(f)
        theta.tofile(f)
    subprocess.run([exe, src, dst], check=True)
    raw = open(dst, "rb").read()
    k = n * m
    A32 = np.frombuffer(raw[: 8 * k]).reshape(n, m)
    fl = np.frombuffer(raw[8 * k : 9 * k], dtype=np.uint8).reshape(n, m)
    A64 = np.frombuffer(raw[9 * k :]).reshape(n, m)
    return A32, fl, A64
