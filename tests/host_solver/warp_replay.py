"""Warp-lockstep replay of the forward kernel's FP32 epoch loop on the benchmark's sweep, from the host
build of the solver headers (measurement infrastructure).

The device runs 8 threads per candidate, each over a run of 250 consecutive epochs, so a warp holds
4 candidates x 8 runs and its 32 lanes solve 32 different epochs side by side. A loop body that a
warp executes costs as long as its busiest lane needs it: a pass of the Aberth loop over a root
that is already done still waits for the lanes that update theirs, and a root slot's polish costs
its slowest lane's Newton steps. This script records, per (candidate, epoch), the passes of the
Aberth loop body, the passes that updated a root, the polish evaluations of each root slot and the
FP32 operations (warp_loop.cpp, with counters planted in a host copy of forward.cuh), maps the
lanes as the kernel does and prints the lanes' mean against the warp's cost per epoch:

    python tests/host_solver/warp_replay.py [--stride 64]

(every stride-th candidate of the 32 populations, all 2000 epochs).
"""
from __future__ import annotations

import argparse
import os
import shutil
import subprocess
import sys
import tempfile

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from host_solver import host_build  # noqa: E402
from paper_1208_4830_gb300 import synth  # noqa: E402

G, SEG = 8, 250  # threads per candidate and epochs per thread of the benchmark's launch

# counters planted in the host copy: (anchor, replacement); each anchor must occur exactly once
HOOKS = [
    ("namespace sblm {", "namespace sblm {\ninline int g_passes, g_updates, g_polish, g_jobs;"),
    ("            if (!(done & 1u)) {\n", "            ++g_passes;\n            if (!(done & 1u)) {\n                ++g_updates;\n"),
    ("            lens_terms(r, zeta, d, q, f, K, qt);\n            if (s == Tol<T>::polish) break;",
     "            lens_terms(r, zeta, d, q, f, K, qt);\n            g_polish += 1 << (3 * i);\n"
     "            if (s == Tol<T>::polish) break;"),
    ("        const int r = aberth(c, z, cap, mask, cold ? Tol<T>::cubic : cubic);",
     "        ++g_jobs;\n        const int r = aberth(c, z, cap, mask, cold ? Tol<T>::cubic : cubic);"),
]


def build(workdir: str) -> str:
    host_build.build(workdir)
    path = os.path.join(workdir, "forward.cuh")
    src = open(path).read()
    for anchor, repl in HOOKS:
        if src.count(anchor) != 1:
            raise RuntimeError(f"anchor not found once in forward.cuh: {anchor[:40]!r}")
        src = src.replace(anchor, repl)
    open(path, "w").write(src)
    shutil.copy(os.path.join(HERE, "count_types.h"), os.path.join(workdir, "count_types.h"))
    exe = os.path.join(workdir, "warp_loop")
    subprocess.run([shutil.which("g++"), "-O2", "-std=c++17", "-I", workdir, os.path.join(HERE, "warp_loop.cpp"),
                    "-o", exe], check=True)
    return exe


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--stride", type=int, default=64)
    a = ap.parse_args()
    sw = synth.forward_sweep(4096, 2000, seed=0)
    thetas = [sw.theta] + [synth.forward_sweep(4096, 16, seed=1000 * k).theta for k in range(1, 32)]
    theta = np.concatenate(thetas)[:: a.stride]
    theta = theta[: (theta.shape[0] // 4) * 4]  # whole warps of 4 candidates
    wd = tempfile.mkdtemp(prefix="sblm_warp_")
    exe = build(wd)
    n, m = theta.shape[0], sw.t.size
    src, dst = os.path.join(wd, "in.bin"), os.path.join(wd, "out.bin")
    with open(src, "wb") as f:
        np.array([n, m, SEG], dtype=np.int32).tofile(f)
        np.ascontiguousarray(sw.t, dtype=np.float64).tofile(f)
        np.ascontiguousarray(theta).tofile(f)
    subprocess.run([exe, src, dst], check=True)
    rec = np.fromfile(dst, dtype=np.int32).reshape(n, m, 6)
    shutil.rmtree(wd, ignore_errors=True)
    # warps: 4 candidates x G runs; at step k lane (c, g) solves epoch g * SEG + k
    W = rec.reshape(n // 4, 4, G, SEG, 6).transpose(0, 3, 1, 2, 4).reshape(n // 4, SEG, 32, 6).astype(np.int64)
    per_slot = np.stack([(W[..., 3] >> (3 * i)) & 7 for i in range(5)], -1)
    print(f"{n} candidates x {m} epochs, {n // 4} warps")
    print(f"FP32 operations per epoch: lane mean {W[..., 0].mean():.1f}")
    print(f"Aberth loop passes per epoch: lane mean {W[..., 1].mean():.2f}, warp {W[..., 1].max(axis=2).mean():.2f}")
    print(f"passes that updated a root: lane mean {W[..., 2].mean():.2f}, warp {W[..., 2].max(axis=2).mean():.2f}")
    print(f"polish evaluations per epoch: lane mean {per_slot.sum(-1).mean():.2f}, "
          f"warp (slowest lane per slot) {per_slot.max(axis=2).sum(-1).mean():.2f}")
    print(f"root-finding jobs per epoch: lane mean {W[..., 4].mean():.3f}; epochs with a MIXED trigger "
          f"{(W[..., 5] != 0).mean():.4f}")


if __name__ == "__main__":
    main()
