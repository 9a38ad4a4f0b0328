"""Algorithmic FP32 / FP64 operations per magnification of the benchmark's forward pass (MIXED),
counted by the host build of the solver with counting types (count_loop.cpp).

The benchmark's step evaluates 32 populations of 4096 sweep candidates on one 2000-epoch
lightcurve in one launch: 131072 candidates, 8 threads per candidate, runs of 250 epochs per
thread (the launch shape the library picks for that size). This script counts every
`--stride`-th candidate of those populations over all epochs with the same runs and prints the
mean operations per magnification:

    python tests/host_solver/count_workload.py [--stride 16] [--seg 250]

With --fp64 --pops 1 --seg 8 it counts the FP64 mode on one population of 4096 candidates (the
launch shape of the benchmark's FP64 context line: 256 threads per candidate, runs of 8 epochs).
"""
from __future__ import annotations

import argparse
import os
import sys
import tempfile

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from host_solver import host_build  # noqa: E402
from oracle import sblm as osb  # noqa: E402
from paper_1208_4830_gb300 import synth  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--stride", type=int, default=16)
    ap.add_argument("--seg", type=int, default=250)
    ap.add_argument("--pops", type=int, default=32)
    ap.add_argument("--fp64", action="store_true", help="count the FP64 mode (every epoch in FP64)")
    a = ap.parse_args()
    sw = synth.forward_sweep(4096, 2000, seed=0)
    thetas = [sw.theta] + [synth.forward_sweep(4096, 16, seed=1000 * k).theta for k in range(1, a.pops)]
    theta = np.concatenate(thetas)[:: a.stride]
    A = osb.magnification(sw.truth[None, :], sw.t)[0]
    sigma = sw.sigma_frac * A
    flux = A + sigma * sw.z
    wd = tempfile.mkdtemp(prefix="sblm_count_")
    host_build.build(wd)
    exe = host_build.build_count(wd)
    n, f32, f64, deferred = host_build.count(exe, theta, sw.t, flux, sigma, a.seg, wd, fp64=a.fp64)
    print(f"rows {theta.shape[0]} epochs {n} runs of {a.seg}: fp32/mag {f32 / n:.1f} fp64/mag {f64 / n:.2f} "
          f"re-solved {deferred / n:.5f} fp64/re-solved epoch {f64 / max(1, deferred):.0f}")


if __name__ == "__main__":
    main()
