"""Benchmark of the population-wide fitness evaluation and EA generation on GB300.

One step = one pass of the whole hot path over one batch: a population of 4096 candidates
(the forward-sweep workload: priors of the sweep, 10% of trajectories aimed through caustics)
evaluated on a 2000-epoch lightcurve (decode, trajectory, quintic, roots, image selection,
magnification, chi^2), then ranked, selected, reproduced and mutated into the next population.
Every step starts from the same population, so the work per step is fixed.

Metric: binary-lens magnifications per second (candidates x epochs per step / step time).
The JSON line also carries the fits/s comparison (unless --no-fits): the learned proposal trained
on the device, then the proposal-seeded MIXED batched fitter, the plain MIXED fitter and the plain
FP64 fitter (each EA + amoeba polish) on held-out synthetic curves, with their success rates.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp32|fp64]
    python bench.py --impl reference ...   # the CPU oracle on the host cores, bounded sample

Under torchrun each rank runs the same workload on its own GPU (weak scaling, no collective on
the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_CAND, N_EP = 4096, 2000
WORKLOAD = "forward sweep: 4096 candidates x 2000 epochs, one EA generation per step"
# gene domains wide enough for every sweep candidate, including the ones re-aimed at caustics
BENCH_LO = np.array([-600.0, 5.0, 0.0, 0.0, 0.3, -4.0])
BENCH_HI = np.array([600.0, 100.0, 3.5, 2.0 * np.pi, 3.0, 0.0])
METRIC = "binary-lens magnifications/s"
UNIT = "magnifications/s"
# FP32 peak of the part: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x maximum SM clock
SMS, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
# executed FP32 arithmetic per magnification of the forward kernel on this workload, from the
# ncu thread-level instruction counts (FMA counted as 2 flop), from the capture summarised in
# profiles/forward_kernel_<precision>_sweep_4096x2000.md. The Aberth sweep has since been rolled
# into a loop over a rotating root array: the same arithmetic in the same amount, so the flop
# count stands, but the capture's DRAM bytes (3.99 MB per launch) belong to the previous build
# and are not reported until the kernel is captured again.
PROFILE = {
    "mixed": {"flop_per_mag": 2973.0, "traffic": None, "file": "profiles/forward_kernel_mixed_sweep_4096x2000.md"},
}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, device):
    """The largest of the ranks' values (every rank gets it); the value itself with one rank."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, step_ms):
    """Units per second of the whole job: every rank's units over the slowest rank's step time."""
    return world * units_per_rank / step_ms * 1e3


def sample_clocks_start(device_index):
    import tempfile

    f = tempfile.NamedTemporaryFile("w", prefix="sblm_clocks_", suffix=".csv", delete=False)
    try:
        p = subprocess.Popen(
            ["nvidia-smi", "-i", str(device_index),
             "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap",
             "--format=csv,noheader,nounits", "-lms", "200"],
            stdout=f, stderr=subprocess.DEVNULL)
        return p, f
    except (OSError, FileNotFoundError):
        f.close()
        os.unlink(f.name)
        return None, None


def sample_clocks_stop(handle):
    p, f = handle
    if p is None:
        return None
    p.terminate()
    try:
        p.wait(timeout=5)
    except subprocess.TimeoutExpired:
        p.kill()
    f.close()
    rows = []
    for line in open(f.name):
        parts = [x.strip() for x in line.split(",")]
        if len(parts) == 6 and parts[0].isdigit():
            rows.append(parts)
    os.unlink(f.name)
    if not rows:
        return None
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for r in rows for i in range(4) if r[2 + i].lower().startswith("active")})
    return {"sm_mhz": statistics.median(int(r[0]) for r in rows), "sm_max_mhz": int(rows[0][1]),
            "reasons": reasons, "samples": len(rows)}


def build_inputs(seed=0):
    from paper_1208_4830_gb300 import synth

    sw = synth.forward_sweep(N_CAND, N_EP, seed=seed)
    a = sw.theta.copy()
    a[:, 5] = np.log10(a[:, 5])
    P0 = (a - BENCH_LO) / (BENCH_HI - BENCH_LO)
    assert np.all((P0 >= 0) & (P0 <= 1)), "sweep candidate outside the bench gene domains"
    return sw, P0


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_1208_4830_gb300 import sblm, synth

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sw, P0 = build_inputs()
    t = torch.tensor(sw.t, device=dev)
    A_true = sblm.magnification(torch.tensor(sw.truth[None, :], device=dev), t, "fp64")[0]
    sigma = float(sw.sigma_frac) * A_true
    flux = A_true + sigma * torch.tensor(sw.z, device=dev)
    P_in = torch.tensor(P0, device=dev)
    step_gpu = make_device_step(sblm, P_in, t, flux, sigma, args.precision, dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    for _ in range(args.warmup):
        step_gpu()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    fwd_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = sample_clocks_start(local)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))  # evict the inputs from L2 between steps (outside the timed events)
        ev[k][0].record(stream)
        step_gpu(fwd_ev[k])
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk = sample_clocks_stop(clocks)
    ms = [a.elapsed_time(b) for a, b in ev]
    fwd_ms = [a.elapsed_time(b) for a, b in fwd_ev]
    step_ms = max_over_ranks(float(np.mean(ms)), dev)

    # end to end through the C ABI with host buffers: pinned host inputs, host results
    e2e = run_e2e(sblm, sw, P0, flux.cpu().numpy(), sigma.cpu().numpy(), args) if args.extras else None

    # the other precisions, same step, for context
    by_prec = {}
    for prec in (("fp64", "fp32", "mixed") if args.extras else ()):
        if prec == args.precision:
            by_prec[prec] = {"ms_per_step": step_ms, "value": N_CAND * N_EP / step_ms * 1e3}
            continue
        st = make_device_step(sblm, P_in, t, flux, sigma, prec, dev)
        st()
        torch.cuda.synchronize()
        n = 2 if prec == "fp64" else 5
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(n):
            st()
        e1.record()
        torch.cuda.synchronize()
        m = e0.elapsed_time(e1) / n
        by_prec[prec] = {"ms_per_step": m, "value": N_CAND * N_EP / m * 1e3}

    fits = run_fits(sblm, args) if (args.extras and args.fits) else None

    if rank == 0:
        value = whole_job_rate(world, N_CAND * N_EP, step_ms)
        fwd = float(np.mean(fwd_ms))
        prof = PROFILE.get(args.precision, {})
        flop = prof.get("flop_per_mag")
        peak = SMS * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
        achieved = flop * N_CAND * N_EP / (fwd * 1e-3) / 1e12 if flop else None
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"mixed": "f32+f64", "fp32": "f32", "fp64": "f64"}[args.precision],
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "candidates": N_CAND, "epochs": N_EP,
                       "precision": args.precision, "l2": "flushed between steps (256 MiB write outside the timed events)",
                       "parallelism": f"replica x{world}" if world > 1 else "1 GPU"},
            "roofline": {"bound": "alu", "kernel": "forward model pass (forward_kernel + MIXED resolve_kernel)",
                         "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None,
                         "traffic": prof.get("traffic"), "kernel_ms": fwd,
                         "flop_per_magnification": flop, "profile": prof.get("file"),
                         "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz (nominal unit counts and clock)"},
            "by_precision": by_prec,
            "fits": fits,
            "e2e": e2e,
            # per step: forward_kernel (+ resolve_kernel in MIXED), rank_kernel, offspring_kernel
            "gpu_launches": (4 if args.precision == "mixed" else 3) * args.steps,
            "clocks": clk,
            "wall_s": wall,
        }
        if args.cpu_baseline and world == 1:
            fh, sh = flux.cpu().numpy(), sigma.cpu().numpy()
            line["cpu_baseline"] = cpu_baseline(sw, fh, sh, args.cpu_seconds)
            try:
                line["cpu_baseline"]["all_cores"] = cpu_baseline_all_cores(sw, fh, sh, line["cpu_baseline"]["value"],
                                                                           args.cpu_seconds)
            except Exception as e:  # the one-core figure stands; report why the pool did not run
                line["cpu_baseline"]["all_cores"] = {"error": f"{type(e).__name__}: {e}"}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def make_device_step(sblm, P_in, t, flux, sigma, precision, dev):
    """One generation through the library: chi^2 of the population from its genes, then the
    operators into a separate buffer (the input population is reused every step)."""
    import ctypes

    import torch

    lib = sblm._lib
    n_pop = P_in.shape[0]
    p = sblm.params(n_pop=n_pop, n_gen=2, precision=precision, seed=0)
    P_out = torch.empty_like(P_in)
    state = sblm.new_state_buffer(dev)
    sblm.ea_init(torch.empty_like(P_in), 6, p, 0, state)
    state0 = state.clone()
    chi = torch.empty(n_pop, dtype=torch.float64, device=dev)
    theta = torch.empty_like(P_in)
    lo, hi = torch.tensor(BENCH_LO, device=dev), torch.tensor(BENCH_HI, device=dev)

    def step(fwd_events=None):
        stream = torch.cuda.current_stream()
        if fwd_events:
            fwd_events[0].record(stream)
        sblm.chi2_genes(P_in, t, flux, sigma, BENCH_LO, BENCH_HI, precision, out=chi)
        if fwd_events:
            fwd_events[1].record(stream)
        P_out.copy_(P_in)
        state.copy_(state0)
        sblm.ea_generation(P_out, chi, p, 0, 0, state)

    return step


# fits: held-out synthetic curves (sweep priors, 10% aimed through caustics, truths inside the fit
# domain), 500 epochs in [-60, 60] d, 2% noise; every arm runs the EA then the amoeba polish
FIT_LCS, FIT_LCS_FP64, FIT_EP, FIT_POP, FIT_GEN, FIT_POLISH = 256, 152, 500, 1024, 150, 2000
# a smaller budget at which the two MIXED arms are also compared (the proposal's gain shows there)
FIT_POP_SMALL, FIT_GEN_SMALL = 512, 150
ISLAND_MIGRATION = 20
PROPOSAL_STEPS, PROPOSAL_BATCH = 1024, 1024  # 1,048,576 training curves
SEED_FRAC = 0.5
# algorithmic flop of one training sample: forward products 2 K N per output position, backward
# the weight and input gradients (the first layer has no input gradient)
CNN_FWD_FLOP = 2 * (256 * 10 * 64 + 128 * 320 * 64 + 64 * 320 * 64 + 32 * 320 * 64 + 2048 * 128 + 128 * 12)
CNN_STEP_FLOP_PER_SAMPLE = 3 * CNN_FWD_FLOP - 2 * 256 * 10 * 64


def _success(best, chi, chi_true, truth, n_ep):
    """Shares of fits meeting: the paper's criterion delta chi^2 / nu < 1 (nu = n_ep - 6, Section
    4.2), delta chi^2 <= 1, and the strict one (paper's criterion and every parameter within 10%:
    t0 relative to tE, alpha relative to 2 pi, the others relative to their own value)."""
    d = chi - chi_true
    da = np.abs((best[:, 3] - truth[:, 3] + np.pi) % (2 * np.pi) - np.pi)
    err = np.stack([np.abs(best[:, 0] - truth[:, 0]) / truth[:, 1], np.abs(best[:, 1] / truth[:, 1] - 1),
                    np.abs(best[:, 2] / truth[:, 2] - 1), da / (2 * np.pi), np.abs(best[:, 4] / truth[:, 4] - 1),
                    np.abs(best[:, 5] / truth[:, 5] - 1)], 1)
    weak = d / (n_ep - 6) < 1
    return {"dchi2_per_dof_lt_1": float(weak.mean()), "dchi2_le_1": float(np.mean(d <= 1.0)),
            "strict": float(np.mean(weak & np.all(err < 0.1, axis=1)))}


def run_fits(sblm, args):
    """Fits per second of the persistent batched fitter (EA + amoeba polish) on held-out curves:
    the proposal-seeded MIXED fitter, the plain MIXED fitter and the plain FP64 fitter, with their
    success rates; and the proposal's training on the device (1M generated curves)."""
    import torch

    from paper_1208_4830_gb300 import synth

    b = synth.heldout_batch(FIT_LCS, seed=77, n_ep=FIT_EP)
    t_d = torch.tensor(b.t, device="cuda")
    A = torch.cat([sblm.magnification(torch.tensor(b.truth[i : i + 1], device="cuda"),
                                      t_d[b.offsets[i] : b.offsets[i + 1]], "fp64")[0] for i in range(FIT_LCS)])
    A = A.cpu().numpy()
    flux, sigma = b.observe(A)
    sl = [slice(b.offsets[i], b.offsets[i + 1]) for i in range(FIT_LCS)]
    chi_true = np.array([sblm.chi2(b.truth[i : i + 1], b.t[s], flux[s], sigma[s], "fp64")[0]
                         for i, s in enumerate(sl)])
    dev = [torch.tensor(x, device="cuda") for x in (b.t, flux, sigma, b.offsets)]

    # the proposal network, trained on the device on curves the forward model generates
    w = sblm.cnn_init(0)
    st = torch.zeros(2 * sblm.cnn_num_params(), device="cuda")
    tp = sblm.cnn_train_params(batch=PROPOSAL_BATCH, n_steps=PROPOSAL_STEPS, warmup=100)
    sblm.cnn_train(w, st, tp, 0, 2)  # graph capture and warm-up (two steps of the schedule)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = sblm.cnn_train(w, st, tp, 2, PROPOSAL_STEPS - 2)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    step_s = train_s / (PROPOSAL_STEPS - 2)
    cnn_flop = CNN_STEP_FLOP_PER_SAMPLE * PROPOSAL_BATCH
    proposal = {
        "training_curves": PROPOSAL_STEPS * PROPOSAL_BATCH, "train_s": train_s + 2 * step_s,
        "curves_per_s": PROPOSAL_BATCH / step_s, "ms_per_step": step_s * 1e3,
        "loss_first": float(np.mean(hist[:10])), "loss_last": float(np.mean(hist[-50:])),
        "step": "generator (priors, forward model FP32, noise, normalisation) + BF16 tensor-core forward and "
                "backward + AdamW, one CUDA graph",
        "tensor_tflops_whole_step": cnn_flop / step_s / 1e12,
        "flop_per_sample": CNN_STEP_FLOP_PER_SAMPLE,
    }

    def arm(precision, frac, n_lc, n_pop=FIT_POP, n_gen=FIT_GEN, n_isl=1):
        d = dev if n_lc == FIT_LCS else [torch.tensor(x, device="cuda") for x in (
            b.t[: b.offsets[n_lc]], flux[: b.offsets[n_lc]], sigma[: b.offsets[n_lc]], b.offsets[: n_lc + 1])]
        p = sblm.params(n_pop=n_pop, n_gen=n_gen, precision=precision, seed=1, polish_fev=FIT_POLISH,
                        n_islands=n_isl, migration_interval=ISLAND_MIGRATION)
        if precision != "fp64":  # graph capture outside the timed call (FP64 is timed once, cold graph)
            sblm.fit_batch_cnn(*d, synth.FIT_LO, synth.FIT_HI, p, w, seed_frac=frac)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        best, chi = sblm.fit_batch_cnn(*d, synth.FIT_LO, synth.FIT_HI, p, w, seed_frac=frac)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        return {"fits_per_s": n_lc / dt, "seconds": dt, "n_lightcurves": n_lc, "n_pop": n_pop, "n_gen": n_gen,
                "n_islands": n_isl,
                "success": _success(best, chi, chi_true[:n_lc], b.truth[:n_lc], FIT_EP),
                "magnifications_per_s": n_isl * n_pop * n_gen * FIT_EP * n_lc / dt}

    out = {"workload": f"held-out synthetic curves (sweep priors, 10% through caustics), {FIT_EP} epochs, "
                       f"2% noise; N_pop {FIT_POP} x {FIT_GEN} generations + amoeba polish ({FIT_POLISH} "
                       f"chi^2 evaluations); batched persistent fitter",
           "success_criterion": "dchi2_per_dof_lt_1 (paper, Section 4.2); dchi2_le_1 and strict also reported",
           "proposal": proposal}
    out["seeded_mixed"] = arm("mixed", SEED_FRAC, FIT_LCS)
    out["plain_mixed"] = arm("mixed", 0.0, FIT_LCS)
    out["plain_fp64"] = arm("fp64", 0.0, FIT_LCS_FP64)
    out["smaller_budget"] = {"seeded_mixed": arm("mixed", SEED_FRAC, FIT_LCS, FIT_POP_SMALL, FIT_GEN_SMALL),
                             "plain_mixed": arm("mixed", 0.0, FIT_LCS, FIT_POP_SMALL, FIT_GEN_SMALL)}
    # the island EA of Section 5.3 at the main arms' budget: 4 populations of N_pop / 4 with a ring
    # migration of their elites every ISLAND_MIGRATION generations
    out["islands_mixed"] = arm("mixed", 0.0, FIT_LCS, FIT_POP // 4, FIT_GEN, n_isl=4)
    out["fits_per_s_seeded_mixed_over_plain_fp64"] = out["seeded_mixed"]["fits_per_s"] / out["plain_fp64"]["fits_per_s"]
    out["paper_workload"] = run_paper_workload(sblm, w)
    out["paper_noisy_blended_workload"] = run_noisy_blended_workload(sblm, w)
    return out


# the paper's own test shape (Section 4.2, noise-free): Table 1 ranges, 100 evenly spaced epochs over
# t0 +- (2..3) tE, sigma 0.01 mag; success per number of peaks, EA + amoeba as in Table 2
PAPER_LCS, PAPER_POP, PAPER_GEN = 256, 1000, 3000
PAPER_TABLE2_EA_AMOEBA = {"1": [97, 100], "2": [98, 100], "3": [97, 98], "4": [94, 94]}  # strict, weak (%)
# the paper's noisy, blended test (Section 4.4): as above with epochs drawn at random, the noise
# model of Section 2.4 (m0 in Table 1's [18, 22]) and a blending fraction f in (0, 1], fitted
# with the blended chi^2 (f profiled out); Table 3 reports EA + amoeba only
PAPER_TABLE3_EA_AMOEBA = {"1": [95, 98], "2": [96, 99], "3": [90, 97], "4": [87, 99]}  # strict, weak (%)


def _peak_classes(sblm, b, n_lc):
    """Peaks of each truth's noise-free source curve over its observing window (3000 samples)."""
    import torch

    from paper_1208_4830_gb300 import synth

    t_d = torch.tensor(b.t, device="cuda")
    A, peaks = [], []
    for i in range(n_lc):
        th = torch.tensor(b.truth[i : i + 1], device="cuda")
        A.append(sblm.magnification(th, t_d[b.offsets[i] : b.offsets[i + 1]], "fp64")[0].cpu().numpy())
        fine = torch.linspace(float(b.t[b.offsets[i]]), float(b.t[b.offsets[i + 1] - 1]), 3000, dtype=torch.float64,
                              device="cuda")
        peaks.append(min(4, synth.count_peaks(sblm.magnification(th, fine, "fp64")[0].cpu().numpy())))
    return np.concatenate(A), np.array(peaks)


def _paper_arms(sblm, w, b, dev, lo, hi, precision, chi_true, nu, peaks, f_true=None):
    """EA + amoeba on the paper-shaped curves, plain and proposal-seeded. Success as in Section 4.2:
    strict = some returned model (every evaluated population, through the device's success
    monitor, or the polished best) has delta chi^2 / nu < 1 and every parameter within 10%; weak =
    the best has delta chi^2 / nu < 1; strict_best_only applies the strict test to the best alone."""
    import torch

    sl = [slice(b.offsets[i], b.offsets[i + 1]) for i in range(len(chi_true))]
    out = {}
    for label, frac in (("plain_mixed", 0.0), ("seeded_mixed", SEED_FRAC)):
        p = sblm.params(n_pop=PAPER_POP, n_gen=PAPER_GEN, precision=precision, seed=1, polish_fev=FIT_POLISH)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        best, chi, first = sblm.fit_batch_monitored(*dev, lo, hi, p, b.truth, chi_true + nu, f_ref=f_true,
                                                    rel_tol=0.1, weights=w, seed_frac=frac)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        tr = b.truth
        da = np.abs((best[:, 3] - tr[:, 3] + np.pi) % (2 * np.pi) - np.pi)
        err = [np.abs(best[:, 0] - tr[:, 0]) / tr[:, 1], np.abs(best[:, 1] / tr[:, 1] - 1),
               np.abs(best[:, 2] / tr[:, 2] - 1), da / (2 * np.pi), np.abs(best[:, 4] / tr[:, 4] - 1),
               np.abs(best[:, 5] / tr[:, 5] - 1)]
        if f_true is not None:
            err.append(np.abs(_fit_f(sblm, best, b, dev, sl) / f_true - 1))
        weak = (chi - chi_true) / nu < 1
        strict_best = weak & np.all(np.stack(err, 1) < 0.1, axis=1)
        strict = strict_best | (first >= 0)

        def pct(x, k=None):
            return round(100 * float((x if k is None else x[peaks == k]).mean()), 1)

        out[label] = {"fits_per_s": len(chi) / dt, "seconds": dt,
                      "success_strict_weak_pct_by_peaks": {str(k): [pct(strict, k), pct(weak, k)] for k in (1, 2, 3, 4)},
                      "success_strict_weak_pct": [pct(strict), pct(weak)],
                      "strict_best_only_pct": pct(strict_best),
                      "median_first_matching_generation": float(np.median(first[first >= 0])) if np.any(first >= 0)
                      else None}
    return out


def _fit_f(sblm, best, b, dev, sl):
    """Profiled blending fraction of each best-fit row (sblm_chi2_blend, FP64)."""
    flux, sigma = dev[1].cpu().numpy(), dev[2].cpu().numpy()
    return np.array([sblm.chi2_blend(best[i : i + 1].copy(), b.t[s], flux[s], sigma[s], "fp64")[1][0]
                     for i, s in enumerate(sl)])


def run_paper_workload(sblm, w):
    import torch

    from paper_1208_4830_gb300 import synth

    b = synth.paper_batch(PAPER_LCS, seed=3)
    A, peaks = _peak_classes(sblm, b, PAPER_LCS)
    flux, sigma = A.copy(), b.sigma(A)
    dev = [torch.tensor(x, device="cuda") for x in (b.t, flux, sigma, b.offsets)]
    out = {"workload": f"{PAPER_LCS} noise-free curves of the paper's test (Table 1 ranges, 100 epochs, sigma 0.01 mag); "
                       f"N_pop {PAPER_POP} x {PAPER_GEN} generations + amoeba ({FIT_POLISH} evaluations)",
           "curves_per_peak_class": {str(k): int(np.sum(peaks == k)) for k in (1, 2, 3, 4)},
           "paper_table2_ea_amoeba_strict_weak_pct": PAPER_TABLE2_EA_AMOEBA}
    # noise-free: the truth's chi^2 is 0; nu = 100 - 6
    out.update(_paper_arms(sblm, w, b, dev, synth.PAPER_LO, synth.PAPER_HI, "mixed", np.zeros(PAPER_LCS), 100 - 6,
                           peaks))
    return out


def run_noisy_blended_workload(sblm, w):
    import torch

    from paper_1208_4830_gb300 import synth

    b = synth.noisy_blended_batch(PAPER_LCS, seed=4)
    A, peaks = _peak_classes(sblm, b, PAPER_LCS)
    flux, sigma = b.observe(A)
    dev = [torch.tensor(x, device="cuda") for x in (b.t, flux, sigma, b.offsets)]
    chi_true = np.array([sblm.chi2_blend(b.truth[i : i + 1].copy(), b.t[b.offsets[i] : b.offsets[i + 1]],
                                         flux[b.offsets[i] : b.offsets[i + 1]], sigma[b.offsets[i] : b.offsets[i + 1]],
                                         "fp64")[0][0] for i in range(PAPER_LCS)])
    out = {"workload": f"{PAPER_LCS} noisy, blended curves of the paper's second test (Table 1 ranges, 100 random "
                       f"epochs, noise model of Section 2.4, f in (0, 1]); blended chi^2 with f profiled out; "
                       f"N_pop {PAPER_POP} x {PAPER_GEN} generations + amoeba ({FIT_POLISH} evaluations)",
           "curves_per_peak_class": {str(k): int(np.sum(peaks == k)) for k in (1, 2, 3, 4)},
           "paper_table3_ea_amoeba_strict_weak_pct": PAPER_TABLE3_EA_AMOEBA}
    # nu = 100 - 7: six lens and trajectory parameters plus f
    out.update(_paper_arms(sblm, w, b, dev, synth.PAPER_LO, synth.PAPER_HI, "mixed+blend", chi_true, 100 - 7, peaks,
                           f_true=b.f))
    return out


def run_e2e(sblm, sw, P0, flux, sigma, args):
    """The same step through the public C ABI with host (pinned) buffers: each step copies the
    population and lightcurve in and the fitness, next population and state out."""
    import torch

    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    P_h, t_h, f_h, s_h = pin(P0), pin(sw.t), pin(flux), pin(sigma)
    chi_h = torch.empty(N_CAND, dtype=torch.float64).pin_memory()
    P_out = torch.empty_like(P_h).pin_memory()
    state = sblm.EAState()
    p = sblm.params(n_pop=N_CAND, n_gen=2, precision=args.precision, seed=0)
    init_P = np.empty_like(P0)
    sblm.ea_init(init_P, 6, p, 0, state)
    import ctypes

    state0 = sblm.EAState.from_buffer_copy(bytes(state))

    def step():
        sblm.chi2_genes(P_h, t_h, f_h, s_h, BENCH_LO, BENCH_HI, args.precision, out=chi_h)
        P_out.copy_(P_h)
        ctypes.memmove(ctypes.addressof(state), ctypes.addressof(state0), ctypes.sizeof(state))
        sblm.ea_generation(P_out, chi_h, p, 0, 0, state)

    for _ in range(max(1, args.warmup)):
        step()
    n = max(3, args.steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n):
        step()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / n
    state_bytes = ctypes.sizeof(sblm.EAState)
    h2d = P0.nbytes + 3 * sw.t.nbytes + P0.nbytes + N_CAND * 8 + state_bytes
    d2h = N_CAND * 8 + P0.nbytes + state_bytes
    return {"value": N_CAND * N_EP / dt, "unit": UNIT, "ms_per_step": dt * 1e3,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "path": "sblm_chi2_genes + sblm_ea_generation on pinned host buffers"}


def oracle_operator_seconds():
    """Seconds the oracle takes for the operators of one generation on the full population."""
    from oracle import ea as oea

    P0 = build_inputs()[1]
    chi = np.random.default_rng(0).uniform(0, 1e4, N_CAND)
    op = oea.EAParams(n_pop=N_CAND, seed=0)
    t0 = time.perf_counter()
    oea.generation(P0, chi, oea.new_state(op), op, 0)
    return time.perf_counter() - t0


def cpu_baseline(sw, flux, sigma, seconds, chunk=16, t_ops=None):
    """The FP64 oracle on the host: chi^2 of as many sweep candidates as fit in about
    `seconds` (in chunks of `chunk`), one process, one thread, plus the operators of one
    generation on the full population (timed here unless `t_ops` is given), amortised per
    magnification."""
    from oracle import sblm as osb

    n_done, t_spent = 0, 0.0
    rows = np.arange(N_CAND)
    k = 0
    while t_spent < seconds and k < N_CAND:
        sel = rows[k : k + chunk]
        t0 = time.perf_counter()
        osb.chi2(sw.theta[sel], sw.t, flux, sigma)
        t_spent += time.perf_counter() - t0
        n_done += sel.size
        k += chunk
    if t_ops is None:
        t_ops = oracle_operator_seconds()
    per_mag = t_spent / (n_done * N_EP) + t_ops / (N_CAND * N_EP)
    return {"value": 1.0 / per_mag, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n_done} of {N_CAND} candidates x {N_EP} epochs (numpy FP64, companion-matrix roots) "
                      f"+ one generation of operators on all {N_CAND} rows, {t_spent + t_ops:.1f} s"}


def _oracle_rows(job):
    """One worker's share of the all-core oracle baseline: the chi^2 of some candidate rows."""
    theta, t, flux, sigma = job
    from oracle import sblm as osb

    osb.chi2(theta, t, flux, sigma)
    return theta.shape[0]


def cpu_baseline_all_cores(sw, flux, sigma, one_core_rate, seconds):
    """The same oracle on every host core: candidate rows spread over one spawned process per
    core (spawned, never forked, after the GPU work), sized from the one-core rate to take about
    `seconds`; the operators of one generation stay on one core as the oracle has them."""
    import multiprocessing as mp

    n = os.cpu_count() or 1
    rows = int(min(N_CAND, max(n, one_core_rate * n * seconds / N_EP)))
    per = -(-rows // (4 * n))  # about four tasks per process
    jobs = [(sw.theta[k : min(rows, k + per)], sw.t, flux, sigma) for k in range(0, rows, per)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(n) as pool:  # leaving the block terminates the workers, also after a timeout
        warm = [(sw.theta[:1], sw.t[:4], flux[:4], sigma[:4])] * n
        pool.map_async(_oracle_rows, warm).get(timeout=300)  # imports, outside the timing
        t0 = time.perf_counter()
        done = sum(pool.map_async(_oracle_rows, jobs).get(timeout=max(120.0, 10 * seconds)))
        wall = time.perf_counter() - t0
    t_ops = oracle_operator_seconds()
    per_mag = wall / (done * N_EP) + t_ops / (N_CAND * N_EP)
    return {"value": 1.0 / per_mag, "unit": UNIT, "cores": n, "kind": "oracle",
            "sample": f"{done} of {N_CAND} candidates x {N_EP} epochs over {n} spawned processes, {wall:.1f} s wall, "
                      f"+ one generation of operators on one core"}


REFERENCE_SECONDS = 120.0


def run_reference(args):
    """The oracle as it stands on the host cores, on the same workload, a bounded sample per step."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    sw, _ = build_inputs()
    from oracle import sblm as osb

    A_true = osb.magnification(sw.truth[None, :], sw.t)[0]
    sigma = sw.sigma_frac * A_true
    flux = A_true + sigma * sw.z
    # the whole run takes about REFERENCE_SECONDS whatever --steps and --warmup are: each step
    # times as many single candidates as fit in its share; the operators are timed once
    per_step = max(0.02, REFERENCE_SECONDS / max(1, args.steps + args.warmup))
    t_ops = oracle_operator_seconds()
    vals = []
    for k in range(args.warmup + args.steps):
        cb = cpu_baseline(sw, flux, sigma, per_step, chunk=1, t_ops=t_ops)
        if k >= args.warmup:
            vals.append(cb["value"])
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": N_CAND * N_EP / value * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "candidates": N_CAND, "epochs": N_EP},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": cb["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp32", "fp64"])
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-fits", dest="fits", action="store_false", help="skip the fits/s measurement")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="skip the end-to-end and other-precision measurements (profiling runs)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
