"""Benchmark of the population-wide fitness evaluation and EA generation on GB300.

One step = one pass of the whole hot path over one batch: 32 independent populations of 4096
candidates each (the forward-sweep workload: priors of the sweep, 10% of trajectories aimed
through caustics), all evaluated on the same 2000-epoch lightcurve in one launch (decode,
trajectory, quintic, roots, image selection, magnification, chi^2), then each population ranked,
selected, reproduced and mutated into its next population (its own Philox stream). Every step
starts from the same populations, so the work per step is fixed: 262M magnifications.

Metric: binary-lens magnifications per second (candidates x epochs per step / step time).
The JSON line also carries (unless --no-fits) the fits/s comparison at the success criterion
delta chi^2 <= 1 against the injected truth: the learned proposal trained on the device, then
the proposal-seeded MIXED batched fitter, the plain MIXED fitter and the plain FP64 fitter (each
EA + amoeba polish) on the same held-out synthetic curves; the seeded and plain MIXED fitters on
2000 held-out curves; the mixed-precision error study (1000 curves); the batched persistent fit of
512 seasonal curves of uneven length (autotuned); and the paper-shaped tests of Tables 2 and 3.

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

N_CAND, N_EP, N_POPS = 4096, 2000, 32
WORKLOAD = ("forward sweep: 32 populations x 4096 candidates x 2000 epochs (one lightcurve), "
            "one EA generation of every population per step")
# gene domains wide enough for every sweep candidate, including the ones re-aimed at caustics
BENCH_LO = np.array([-600.0, 5.0, 0.0, 0.0, 0.3, -4.0])
BENCH_HI = np.array([600.0, 100.0, 8.0, 2.0 * np.pi, 3.0, 0.0])
METRIC = "binary-lens magnifications/s"
UNIT = "magnifications/s"
FP32_LANES = 128  # FP32 FMA lanes per SM (Blackwell)
# algorithmic FP32 (and FP64) arithmetic per magnification of this workload's launch shape, counted
# by the host build of the solver on a sample of the sweep (tests/host_solver: every floating-point
# operation the algorithm performs as written, a fused multiply-add counted as 2); see
# profiles/forward_kernel_mixed_sweep_32x4096x2000.md
# (python tests/host_solver/count_workload.py --stride 16 --seg 250: 8192 of the 131072 candidates, every
# epoch; 0.341% of the epochs re-solved in FP64, 3087 FP64 operations each). traffic: DRAM bytes
# read + written per forward_kernel launch of the full step, from an ncu capture of 20 populations
# scaled by the magnifications (the dense term rows, 8 B per magnification, and register spills)
FLOP_COUNT = {"mixed": {"fp32_per_mag": 2387.8, "fp64_per_mag": 10.51, "traffic": 3.58e9,
                        "file": "profiles/forward_kernel_mixed_sweep_32x4096x2000.md"}}
# the FP64 mode on one population of 4096 (256 threads per candidate, runs of 8 epochs): FP64
# operations per magnification, counted the same way
# (python tests/host_solver/count_workload.py --fp64 --pops 1 --stride 16 --seg 8)
FP64_CONTEXT_FLOP_PER_MAG = 3416.4


def set_populations(n):
    """Populations per step (the workload description follows)."""
    global N_POPS, WORKLOAD
    N_POPS = int(n)
    WORKLOAD = (f"forward sweep: {N_POPS} populations x {N_CAND} candidates x {N_EP} epochs (one lightcurve), "
                f"one EA generation of every population per step")


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
    """The sweep lightcurve (epochs and truth of sweep `seed`) and N_POPS populations of sweep
    candidates (sweeps seed, seed + 1000, ...; each 10% aimed through caustics) as genes."""
    from paper_1208_4830_gb300 import synth

    sw = synth.forward_sweep(N_CAND, N_EP, seed=seed)
    thetas = [sw.theta] + [synth.forward_sweep(N_CAND, 16, seed=seed + 1000 * k).theta for k in range(1, N_POPS)]
    theta = np.concatenate(thetas)
    a = theta.copy()
    a[:, 5] = np.log10(a[:, 5])
    P0 = (a - BENCH_LO) / (BENCH_HI - BENCH_LO)
    assert np.all((P0 >= 0) & (P0 <= 1)), "sweep candidate outside the bench gene domains"
    return sw, theta, P0


def pipe_time_fraction(fp32_flop, fp64_flop, fp32_peak_tflops, fp64_peak_tflops, seconds):
    """The time the FP32 and FP64 pipes would need for the given algorithmic work at their peak
    rates, as a fraction of the measured time: the roofline fraction of a pass whose work is split
    between the two pipes (an FP64 operation costs the FP32 pipe's rate / the FP64 pipe's rate as
    much time as an FP32 one)."""
    return (fp32_flop / (fp32_peak_tflops * 1e12) + fp64_flop / (fp64_peak_tflops * 1e12)) / seconds


def measured_peaks(sblm, device_index, clk):
    """FP32 / FP64 peaks of this device: nominal (SMs x lanes x 2 flop x maximum SM clock) and
    measured (sblm_peak_rates: FMA chains on every SM)."""
    import torch

    sms = torch.cuda.get_device_properties(device_index).multi_processor_count
    mhz = (clk or {}).get("sm_max_mhz")
    if not mhz:
        try:
            mhz = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"]
        except (OSError, ValueError, KeyError):
            mhz = 2070.0
    fp32_m, fp64_m = sblm.peak_rates()
    return {"sms": sms, "sm_max_mhz": float(mhz), "fp32_nominal": sms * FP32_LANES * 2 * float(mhz) * 1e6 / 1e12,
            "fp32_measured": fp32_m, "fp64_measured": fp64_m}


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_1208_4830_gb300 import sblm

    t_start = time.perf_counter()
    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sw, _, P0 = build_inputs()
    t = torch.tensor(sw.t, device=dev)
    A_true = sblm.magnification(torch.tensor(sw.truth[None, :], device=dev), t, "fp64")[0]
    sigma = float(sw.sigma_frac) * A_true
    flux = A_true + sigma * torch.tensor(sw.z, device=dev)
    P_in = torch.tensor(P0, device=dev)
    step_gpu = make_device_step(sblm, P_in, t, flux, sigma, args.precision, dev, N_POPS)
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
    mags = N_POPS * N_CAND * N_EP

    # end to end through the C ABI with host buffers: pinned host inputs, host results
    e2e = run_e2e(sblm, sw, P0, flux.cpu().numpy(), sigma.cpu().numpy(), args) if args.extras else None

    # the other precisions for context: FP32 on the same step, FP64 on one population of 4096
    by_prec = {}
    for prec in (("fp64", "fp32", "mixed") if args.extras else ()):
        if prec == args.precision:
            by_prec[prec] = {"ms_per_step": step_ms, "value": mags / step_ms * 1e3, "populations": N_POPS}
            continue
        n_p = 1 if prec == "fp64" else N_POPS
        st = make_device_step(sblm, P_in[: n_p * N_CAND].contiguous(), t, flux, sigma, prec, dev, n_p)
        st()
        torch.cuda.synchronize()
        n = 3
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(n):
            st()
        e1.record()
        torch.cuda.synchronize()
        m = e0.elapsed_time(e1) / n
        by_prec[prec] = {"ms_per_step": m, "value": n_p * N_CAND * N_EP / m * 1e3, "populations": n_p}
        if prec == "fp64":  # the FP64 forward model against the FP64 pipe's measured rate
            by_prec[prec]["fp64_flop_per_magnification"] = FP64_CONTEXT_FLOP_PER_MAG
            by_prec[prec]["achieved_fp64_tflops"] = FP64_CONTEXT_FLOP_PER_MAG * n_p * N_CAND * N_EP / (m * 1e-3) / 1e12

    peaks = measured_peaks(sblm, local, clk) if rank == 0 else None
    if peaks and "fp64" in by_prec:
        by_prec["fp64"]["frac_of_measured_fp64_rate"] = by_prec["fp64"]["achieved_fp64_tflops"] / peaks["fp64_measured"]
    fits = None
    if args.extras and args.fits and world == 1:  # the fit workloads run on one GPU only
        fits = run_fits(sblm, args, deadline=t_start + args.time_budget, peaks=peaks)

    if rank == 0:
        value = whole_job_rate(world, mags, step_ms)
        fwd = float(np.mean(fwd_ms))
        fc = FLOP_COUNT.get(args.precision, {})
        f32 = fc.get("fp32_per_mag")
        achieved = f32 * mags / (fwd * 1e-3) / 1e12 if f32 else None
        peak = peaks["fp32_nominal"]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"mixed": "f32+f64", "fp32": "f32", "fp64": "f64"}[args.precision],
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "populations": N_POPS, "candidates": N_CAND, "epochs": N_EP,
                       "magnifications_per_step": mags, "precision": args.precision,
                       "l2": "flushed between steps (256 MiB write outside the timed events)",
                       "parallelism": f"replica x{world}" if world > 1 else "1 GPU"},
            "roofline": {"bound": "alu", "kernel": "forward model pass (forward_kernel + MIXED resolve_kernel and "
                                                  "term_sum_kernel)",
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": (achieved / peak) if achieved else None,
                         "frac_of_measured_fma_rate": (achieved / peaks["fp32_measured"]) if achieved else None,
                         "frac_pipe_time": pipe_time_fraction(f32 * mags, fc.get("fp64_per_mag", 0.0) * mags, peak,
                                                              peaks["fp64_measured"], fwd * 1e-3) if f32 else None,
                         "frac_pipe_time_note": "(FP32 work / FP32 peak + FP64 re-solve work / measured FP64 rate) "
                                                "/ forward-pass time",
                         "traffic": fc.get("traffic"), "kernel_ms": fwd,
                         "fp32_flop_per_magnification": f32, "fp64_flop_per_magnification": fc.get("fp64_per_mag"),
                         "flop_count": "algorithmic: every FP32 operation of the solver as written, counted by the "
                                       "host build on this launch shape (FMA = 2)",
                         "profile": fc.get("file"),
                         "peak_source": f"{peaks['sms']} SMs x {FP32_LANES} FP32 lanes x 2 flop x "
                                        f"{peaks['sm_max_mhz']:.0f} MHz (device query and maximum SM clock); "
                                        f"measured FMA-chain rate {peaks['fp32_measured']:.1f} TFLOP/s"},
            "peaks": peaks,
            "by_precision": by_prec,
            "fits": fits,
            "e2e": e2e,
            # per step: forward_kernel (+ resolve_kernel and term_sum_kernel in MIXED), then one
            # rank_kernel and one offspring_kernel for all populations
            "gpu_launches": ((3 if args.precision == "mixed" else 1) + 2) * args.steps,
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
        line["bench_wall_s"] = time.perf_counter() - t_start
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def make_device_step(sblm, P_in, t, flux, sigma, precision, dev, n_pops):
    """One generation of n_pops populations through the library: the chi^2 of every population's
    rows from their genes in one call, then the operators of all populations in one call (each its
    own stream id) on a copy (the input populations are reused every step)."""
    import torch

    p = sblm.params(n_pop=N_CAND, n_gen=2, precision=precision, seed=0)
    P_out = torch.empty_like(P_in)
    states = torch.stack([sblm.new_state_buffer(dev) for _ in range(n_pops)])
    for k in range(n_pops):
        sblm.ea_init(torch.empty_like(P_in[:N_CAND]), 6, p, k, states[k])
    states0 = states.clone()
    chi = torch.empty(n_pops * N_CAND, dtype=torch.float64, device=dev)

    def step(fwd_events=None):
        stream = torch.cuda.current_stream()
        if fwd_events:
            fwd_events[0].record(stream)
        sblm.chi2_genes(P_in, t, flux, sigma, BENCH_LO, BENCH_HI, precision, out=chi)
        if fwd_events:
            fwd_events[1].record(stream)
        P_out.copy_(P_in)
        states.copy_(states0)
        sblm.ea_generation_batch(P_out, chi, p, 0, 0, states)  # population k on stream id k

    return step


# fits: held-out synthetic curves (sweep priors, 10% aimed through caustics, truths inside the fit
# domain), 500 epochs in [-60, 60] d, 2% noise; every arm runs the EA then the amoeba polish. The
# fits/s comparison uses the same curves in every arm (the first HEAD_LCS, one per SM) and a
# budget at which the arms reach 90% success at delta chi^2 <= 1; the MIXED arms also fit all
# BIG_LCS held-out curves
HEAD_LCS, BIG_LCS, FIT_EP, FIT_POP, FIT_GEN, FIT_POLISH = 152, 2000, 500, 1024, 1200, 2000
# the amoeba runs from the 8 fittest distinct solutions of each fit (distinct: some gene differs by
# more than 0.05) and keeps the best; the paper polishes the fittest only (polish_starts 1)
FIT_STARTS, FIT_RADIUS = 8, 0.05
PROPOSAL_STEPS, PROPOSAL_BATCH = 1024, 1024  # 1,048,576 training curves
SEED_FRAC = 0.5
# mixed-precision error study: the first 1000 held-out curves (500 epochs at 2% noise)
ERR_LCS = 1000
# batched persistent fit of seasonal curves of uneven length (200-5000 epochs, 120-day gaps,
# sigma 0.5-5%), N_pop 1024 x 300 generations, one graph-captured launch, autotuned launch shape
SEASON_LCS, SEASON_POP, SEASON_GEN = 512, 1024, 300
# algorithmic flop of one training sample: forward products 2 K N per output position, backward
# the weight and input gradients (the first layer has no input gradient)
CNN_FWD_FLOP = 2 * (256 * 10 * 64 + 128 * 320 * 64 + 64 * 320 * 64 + 32 * 320 * 64 + 2048 * 128 + 128 * 12)
CNN_STEP_FLOP_PER_SAMPLE = 3 * CNN_FWD_FLOP - 2 * 256 * 10 * 64


def _success(best, chi, chi_true, truth, n_ep):
    """Shares of fits meeting: delta chi^2 <= 1 against the injected truth (the criterion the
    comparison is judged by), the paper's delta chi^2 / nu < 1 (nu = n_ep - 6, Section 4.2), and
    the strict one (paper's criterion and every parameter within 10%: t0 relative to tE, alpha
    relative to 2 pi, the others relative to their own value); with the binomial standard error
    of the first."""
    d = chi - chi_true
    da = np.abs((best[:, 3] - truth[:, 3] + np.pi) % (2 * np.pi) - np.pi)
    err = np.stack([np.abs(best[:, 0] - truth[:, 0]) / truth[:, 1], np.abs(best[:, 1] / truth[:, 1] - 1),
                    np.abs(best[:, 2] / truth[:, 2] - 1), da / (2 * np.pi), np.abs(best[:, 4] / truth[:, 4] - 1),
                    np.abs(best[:, 5] / truth[:, 5] - 1)], 1)
    weak = d / (n_ep - 6) < 1
    ok = float(np.mean(d <= 1.0))
    return {"dchi2_le_1": ok, "dchi2_le_1_stderr": float(np.sqrt(ok * (1 - ok) / max(1, d.size))),
            "dchi2_per_dof_lt_1": float(weak.mean()), "strict": float(np.mean(weak & np.all(err < 0.1, axis=1)))}


class Budget:
    """Wall-clock budget of the optional measurements: a section runs only if its estimated
    duration fits in what is left (it is then reported as skipped)."""

    def __init__(self, deadline):
        self.deadline = deadline

    def left(self):
        return self.deadline - time.perf_counter()

    def run(self, out, key, estimate_s, fn):
        if self.left() < estimate_s:
            out[key] = {"skipped": f"time budget: ~{estimate_s:.0f} s needed, {max(0.0, self.left()):.0f} s left"}
            return None
        try:
            out[key] = fn()
        except Exception as e:  # a failed section is reported, the others still run
            out[key] = {"error": f"{type(e).__name__}: {e}"}
        return out[key]


def _heldout(sblm, n_lc):
    """The held-out curves with observed flux, sigma and the FP64 chi^2 of their truths."""
    import torch

    from paper_1208_4830_gb300 import synth

    b = synth.heldout_batch(n_lc, seed=77, n_ep=FIT_EP)
    t_d = torch.tensor(b.t, device="cuda")
    A = torch.cat([sblm.magnification(torch.tensor(b.truth[i : i + 1], device="cuda"),
                                      t_d[b.offsets[i] : b.offsets[i + 1]], "fp64")[0] for i in range(n_lc)])
    flux, sigma = b.observe(A.cpu().numpy())
    chi_true = np.empty(n_lc)
    f_d, s_d = torch.tensor(flux, device="cuda"), torch.tensor(sigma, device="cuda")
    for i in range(n_lc):
        sl = slice(int(b.offsets[i]), int(b.offsets[i + 1]))
        chi_true[i] = float(sblm.chi2(torch.tensor(b.truth[i : i + 1], device="cuda"), t_d[sl], f_d[sl], s_d[sl],
                                      "fp64")[0])
    return b, flux, sigma, chi_true


def run_fits(sblm, args, deadline, peaks):
    """The fits/s comparison at delta chi^2 <= 1 and the batched-fitter workloads, each section
    within the wall-clock budget (see Budget)."""
    import torch

    from paper_1208_4830_gb300 import synth

    budget = Budget(deadline)
    out = {"success_criterion": "dchi2_le_1 (delta chi^2 <= 1 against the injected truth); the paper's "
                                "dchi2_per_dof_lt_1 (Section 4.2) and strict also reported",
           "budget_s": args.time_budget}
    b, flux, sigma, chi_true = _heldout(sblm, BIG_LCS)
    dev_all = [torch.tensor(x, device="cuda") for x in (b.t, flux, sigma, b.offsets)]

    def subset(n):
        e = int(b.offsets[n])
        return [torch.tensor(x, device="cuda") for x in (b.t[:e], flux[:e], sigma[:e], b.offsets[: n + 1])]

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
    out["proposal"] = {
        "training_curves": PROPOSAL_STEPS * PROPOSAL_BATCH, "train_s": train_s + 2 * step_s,
        "curves_per_s": PROPOSAL_BATCH / step_s, "ms_per_step": step_s * 1e3,
        "loss_first": float(np.mean(hist[:10])), "loss_last": float(np.mean(hist[-50:])),
        "step": "generator (priors, forward model FP32, noise, normalisation) + BF16 tensor-core forward and "
                "backward + AdamW, one CUDA graph",
        "tensor_tflops_whole_step": CNN_STEP_FLOP_PER_SAMPLE * PROPOSAL_BATCH / step_s / 1e12,
        "flop_per_sample": CNN_STEP_FLOP_PER_SAMPLE,
    }

    def arm(precision, frac, n_lc, n_gen=FIT_GEN, repeat=False):
        """One timed fit of the first n_lc curves, graph capture included (the same procedure for
        every arm; `repeat` times a second, warm call as well)."""
        d = dev_all if n_lc == BIG_LCS else subset(n_lc)
        p = sblm.params(n_pop=FIT_POP, n_gen=n_gen, precision=precision, seed=1, polish_fev=FIT_POLISH,
                        polish_starts=FIT_STARTS, polish_radius=FIT_RADIUS)
        times = []
        for _ in range(2 if repeat else 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            best, chi = sblm.fit_batch_cnn(*d, synth.FIT_LO, synth.FIT_HI, p, w, seed_frac=frac)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        dt = times[0]
        r = {"fits_per_s": n_lc / dt, "seconds": dt, "n_lightcurves": n_lc, "n_pop": FIT_POP, "n_gen": n_gen,
             "polish_fev": FIT_POLISH, "polish_starts": FIT_STARTS,
             "success": _success(best, chi, chi_true[:n_lc], b.truth[:n_lc], FIT_EP),
             "magnifications_per_s": FIT_POP * n_gen * FIT_EP * n_lc / dt, "timing": "first call (graph capture "
                                                                                      "included)"}
        if repeat:
            r["seconds_warm"] = times[1]
        return r, best, chi

    # 1. the comparison: the same curves, the same budget, seeded MIXED vs plain MIXED vs plain FP64
    head = {"workload": f"first {HEAD_LCS} held-out curves (one per SM): sweep priors, 10% through caustics, "
                        f"{FIT_EP} epochs, 2% noise; N_pop {FIT_POP} x {FIT_GEN} generations + amoeba polish "
                        f"({FIT_POLISH} chi^2 evaluations from each of the {FIT_STARTS} fittest distinct solutions); "
                        f"batched persistent fitter"}
    out["head_to_head"] = head
    fits, head_best = {}, {}
    for key, prec, frac, est in (("seeded_mixed", "mixed", SEED_FRAC, 60), ("plain_mixed", "mixed", 0.0, 60),
                                 ("plain_fp64", "fp64", 0.0, 860)):
        def go(prec=prec, frac=frac, key=key):
            r, best, _ = arm(prec, frac, HEAD_LCS)
            head_best[key] = best
            return r
        r = budget.run(head, key, est, go)
        if r and "fits_per_s" in r:
            fits[key] = r
    if "seeded_mixed" in fits and "plain_fp64" in fits:
        ok = all(fits[k]["success"]["dchi2_le_1"] >= 0.9 for k in ("seeded_mixed", "plain_fp64"))
        head["fits_per_s_seeded_mixed_over_plain_fp64"] = fits["seeded_mixed"]["fits_per_s"] / fits["plain_fp64"]["fits_per_s"]
        head["both_at_least_90pct_dchi2_le_1"] = ok
    if "plain_mixed" in fits and "plain_fp64" in fits:
        head["fits_per_s_plain_mixed_over_plain_fp64"] = fits["plain_mixed"]["fits_per_s"] / fits["plain_fp64"]["fits_per_s"]

    # mixed-precision error against FP64 on the first 1000 curves: every magnification and chi^2 at
    # the truths (and at the plain MIXED fits' bests of the first 152), and the success of the MIXED
    # and FP64 fits of the comparison
    def error_study():
        n = ERR_LCS
        rel_A, rel_c, abs_c = [], [], []
        best = head_best.get("plain_mixed")
        t_d = dev_all[0]
        for i in range(n):
            sl = slice(int(b.offsets[i]), int(b.offsets[i + 1]))
            rows = b.truth[i : i + 1] if best is None or i >= len(best) else np.vstack([b.truth[i : i + 1],
                                                                                      best[i : i + 1]])
            th = torch.tensor(rows, device="cuda")
            a64 = sblm.magnification(th, t_d[sl], "fp64")
            amx = sblm.magnification(th, t_d[sl], "mixed")
            rel_A.append(((amx - a64).abs() / a64).flatten().cpu().numpy())
            c64 = sblm.chi2(th, t_d[sl], dev_all[1][sl], dev_all[2][sl], "fp64")
            cmx = sblm.chi2(th, t_d[sl], dev_all[1][sl], dev_all[2][sl], "mixed")
            rel_c.append(((cmx - c64).abs() / c64).cpu().numpy())
            abs_c.append((cmx - c64).abs().cpu().numpy())
        rel_A, rel_c, abs_c = np.concatenate(rel_A), np.concatenate(rel_c), np.concatenate(abs_c)
        r = {"workload": f"first {n} held-out curves ({FIT_EP} epochs, 2% noise): every epoch of each truth, "
                         f"and of the plain MIXED fits' bests of the first {HEAD_LCS}",
             "magnification_rel_err": {"values": int(rel_A.size), "median": float(np.median(rel_A)),
                                       "max": float(rel_A.max()), "p999": float(np.quantile(rel_A, 0.999))},
             "chi2_rel_err": {"median": float(np.median(rel_c)), "max": float(rel_c.max())},
             "chi2_abs_err": {"median": float(np.median(abs_c)), "max": float(abs_c.max())}}
        if "plain_fp64" in fits:
            r["success_fp64_dchi2_le_1_first_152"] = fits["plain_fp64"]["success"]["dchi2_le_1"]
            r["success_mixed_dchi2_le_1_first_152"] = fits.get("plain_mixed", {}).get("success", {}).get("dchi2_le_1")
        return r

    budget.run(out, "mixed_precision_error", 40, error_study)
    budget.run(out, "seasonal_batch", 150, lambda: run_seasonal(sblm))
    # all 2000 held-out curves (the learned proposal's held-out test): seeded vs plain MIXED
    big = {"workload": f"{BIG_LCS} held-out curves, same recipe and budget"}
    out["heldout_2000"] = big
    res = {}
    for key, frac in (("seeded_mixed", SEED_FRAC), ("plain_mixed", 0.0)):
        def go(frac=frac, key=key):
            r, best, chi = arm("mixed", frac, BIG_LCS)
            res[key] = (best, chi)
            return r
        budget.run(big, key, 520, go)
    if len(res) == 2:
        ok_s = (res["seeded_mixed"][1] - chi_true) <= 1.0
        ok_p = (res["plain_mixed"][1] - chi_true) <= 1.0
        dlt = ok_s.astype(float) - ok_p.astype(float)
        big["seeded_minus_plain_dchi2_le_1"] = float(dlt.mean())
        big["seeded_minus_plain_stderr"] = float(dlt.std(ddof=1) / np.sqrt(dlt.size))

    budget.run(out, "paper_workload", 90, lambda: run_paper_workload(sblm, w))
    budget.run(out, "paper_noisy_blended_workload", 90, lambda: run_noisy_blended_workload(sblm, w))
    # the same noisy test at a longer budget (the paper's budget was 20 minutes per fit)
    budget.run(out, "paper_noisy_blended_workload_long", 300,
               lambda: run_noisy_blended_workload(sblm, w, n_gen=PAPER_GEN_LONG))
    return out


def run_seasonal(sblm):
    """512 seasonal curves of uneven length in one graph-captured persistent launch per fit, with the
    launch shape picked by the autotuner (tuned on this workload, a fresh cache)."""
    import tempfile

    import torch

    from paper_1208_4830_gb300 import synth

    b = synth.seasonal_batch(SEASON_LCS, seed=0)
    t_d = torch.tensor(b.t, device="cuda")
    A = torch.cat([sblm.magnification(torch.tensor(b.truth[i : i + 1], device="cuda"),
                                      t_d[b.offsets[i] : b.offsets[i + 1]], "fp64")[0] for i in range(SEASON_LCS)])
    flux, sigma = b.observe(A.cpu().numpy())
    d = [t_d] + [torch.tensor(x, device="cuda") for x in (flux, sigma, b.offsets)]
    p = sblm.params(n_pop=SEASON_POP, n_gen=SEASON_GEN, precision="mixed", seed=1)
    cache = os.path.join(tempfile.mkdtemp(prefix="sblm_tune_"), "tune.json")
    t0 = time.perf_counter()
    tuning = sblm.autotune_batch(*d, synth.FIT_LO, synth.FIT_HI, p, trial_generations=2, cache=cache)
    tune_s = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    best, chi = sblm.fit_batch(*d, synth.FIT_LO, synth.FIT_HI, p, tuning=tuning)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    n_ep = np.diff(b.offsets)
    mags = SEASON_POP * SEASON_GEN * int(n_ep.sum())
    chi_true = np.array([float(sblm.chi2(b.truth[i : i + 1], b.t[b.offsets[i] : b.offsets[i + 1]],
                                         flux[b.offsets[i] : b.offsets[i + 1]], sigma[b.offsets[i] : b.offsets[i + 1]],
                                         "fp64")[0]) for i in range(SEASON_LCS)])
    return {"workload": f"{SEASON_LCS} seasonal curves of {int(n_ep.min())}-{int(n_ep.max())} epochs "
                        f"({int(n_ep.sum())} in all; 245-day seasons, 120-day gaps, sigma 0.5-5%), N_pop "
                        f"{SEASON_POP} x {SEASON_GEN} generations, MIXED, one graph-captured persistent launch",
            "tuning": {"group": int(tuning.group), "block": int(tuning.block), "autotune_s": tune_s},
            "fits_per_s": SEASON_LCS / dt, "seconds": dt, "magnifications_per_s": mags / dt,
            "magnifications": mags, "success_dchi2_le_1": float(np.mean(chi - chi_true <= 1.0))}


# the paper's own test shape (Section 4.2, noise-free): Table 1 ranges, 100 evenly spaced epochs over
# t0 +- (2..3) tE, sigma 0.01 mag; success per number of peaks, EA + amoeba as in Table 2
PAPER_LCS, PAPER_POP, PAPER_GEN = 256, 1000, 3000
PAPER_GEN_LONG = 10000
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


def _paper_arms(sblm, w, b, dev, lo, hi, precision, chi_true, nu, peaks, f_true=None, m0=None, n_gen=None):
    """EA + amoeba on the paper-shaped curves, plain and proposal-seeded. Success as in Section 4.2:
    strict = some returned model (every evaluated population, through the device's success
    monitor, or the polished best) has delta chi^2 / nu < 1 and every parameter within 10%; weak =
    the best has delta chi^2 / nu < 1; strict_best_only applies the strict test to the best alone."""
    import torch

    sl = [slice(b.offsets[i], b.offsets[i + 1]) for i in range(len(chi_true))]
    out = {}
    for label, frac in (("plain_mixed", 0.0), ("seeded_mixed", SEED_FRAC)):
        p = sblm.params(n_pop=PAPER_POP, n_gen=n_gen or PAPER_GEN, precision=precision, seed=1, polish_fev=FIT_POLISH)
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
        # the same errors relative to each parameter's range of Table 1 (a looser reading of "errors in
        # all fitted parameters < 10%"; alpha on 2 pi, q linear as in the paper's encoding)
        span = np.array(hi) - np.array(lo)
        err_r = [np.abs(best[:, 0] - tr[:, 0]) / span[0], np.abs(best[:, 1] - tr[:, 1]) / span[1],
                 np.abs(best[:, 2] - tr[:, 2]) / span[2], da / (2 * np.pi), np.abs(best[:, 4] - tr[:, 4]) / span[4],
                 np.abs(best[:, 5] - tr[:, 5]) / (10.0 ** hi[5] - 10.0 ** lo[5])]
        if f_true is not None:
            f_fit = _fit_f(sblm, best, b, dev, sl)
            err.append(np.abs(f_fit / f_true - 1))
            err_r.append(np.abs(f_fit - f_true))
        weak = (chi - chi_true) / nu < 1
        strict_best = weak & np.all(np.stack(err, 1) < 0.1, axis=1)
        strict_range = weak & np.all(np.stack(err_r, 1) < 0.1, axis=1)
        strict = strict_best | (first >= 0)

        def pct(x, k=None):
            return round(100 * float((x if k is None else x[peaks == k]).mean()), 1)

        out[label] = {"fits_per_s": len(chi) / dt, "seconds": dt,
                      "success_strict_weak_pct_by_peaks": {str(k): [pct(strict, k), pct(weak, k)] for k in (1, 2, 3, 4)},
                      "success_strict_weak_pct": [pct(strict), pct(weak)],
                      "strict_best_only_pct": pct(strict_best),
                      "strict_best_only_range_relative_pct_by_peaks": {str(k): pct(strict_range, k) for k in (1, 2, 3, 4)},
                      "median_first_matching_generation": float(np.median(first[first >= 0])) if np.any(first >= 0)
                      else None}
        if m0 is not None:  # the noisy test's success against the source's unlensed magnitude
            bins = ((18.0, 19.0), (19.0, 20.0), (20.0, 21.0), (21.0, 22.0))
            out[label]["success_strict_weak_pct_by_m0"] = {
                f"{a:g}-{z:g}": [round(100 * float(strict[(m0 >= a) & (m0 < z)].mean()), 1),
                                 round(100 * float(weak[(m0 >= a) & (m0 < z)].mean()), 1)] for a, z in bins}
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


def run_noisy_blended_workload(sblm, w, n_gen=None):
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
                       f"epochs, noise model of Section 2.4 at the true magnitude, m0 the source's unlensed magnitude in "
                       f"[18, 22], f in (0, 1]); blended chi^2 with f profiled out; "
                       f"N_pop {PAPER_POP} x {n_gen or PAPER_GEN} generations + amoeba ({FIT_POLISH} evaluations)",
           "curves_per_peak_class": {str(k): int(np.sum(peaks == k)) for k in (1, 2, 3, 4)},
           "paper_table3_ea_amoeba_strict_weak_pct": PAPER_TABLE3_EA_AMOEBA}
    # nu = 100 - 7: six lens and trajectory parameters plus f
    out.update(_paper_arms(sblm, w, b, dev, synth.PAPER_LO, synth.PAPER_HI, "mixed+blend", chi_true, 100 - 7, peaks,
                           f_true=b.f, m0=b.m0, n_gen=n_gen))
    return out


def run_e2e(sblm, sw, P0, flux, sigma, args):
    """The same step through the public C ABI with host (pinned) buffers: each step copies the
    populations and lightcurve in and the fitness, next populations and states out."""
    import ctypes

    import torch

    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    P_h, t_h, f_h, s_h = pin(P0), pin(sw.t), pin(flux), pin(sigma)
    n = P0.shape[0]
    chi_h = torch.empty(n, dtype=torch.float64).pin_memory()
    P_out = torch.empty_like(P_h).pin_memory()
    p = sblm.params(n_pop=N_CAND, n_gen=2, precision=args.precision, seed=0)
    states, states0 = [], []
    for k in range(N_POPS):
        st = sblm.EAState()
        sblm.ea_init(np.empty((N_CAND, 6)), 6, p, k, st)
        states.append(st)
        states0.append(bytes(st))

    def step():
        sblm.chi2_genes(P_h, t_h, f_h, s_h, BENCH_LO, BENCH_HI, args.precision, out=chi_h)
        P_out.copy_(P_h)
        for k in range(N_POPS):
            ctypes.memmove(ctypes.addressof(states[k]), states0[k], len(states0[k]))
        sblm.ea_generation_batch(P_out, chi_h, p, 0, 0, states)

    for _ in range(max(1, min(args.warmup, 2))):
        step()
    reps = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        step()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / reps
    state_bytes = ctypes.sizeof(sblm.EAState)
    # in: populations and lightcurve for the chi^2, then per population its rows, chi^2 and state;
    # out: the chi^2, then per population its next rows and state
    h2d = P0.nbytes + 3 * sw.t.nbytes + P0.nbytes + n * 8 + N_POPS * state_bytes
    d2h = n * 8 + P0.nbytes + N_POPS * state_bytes
    return {"value": N_POPS * N_CAND * N_EP / dt, "unit": UNIT, "ms_per_step": dt * 1e3, "steps": reps,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "path": "sblm_chi2_genes + sblm_ea_generation_batch (32 populations) on pinned host buffers"}


def oracle_operator_seconds():
    """Seconds the oracle takes for the operators of one generation on the full population."""
    from oracle import ea as oea

    P0 = build_inputs()[2][:N_CAND]
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
                      f"+ one generation of operators on all {N_CAND} rows, {t_spent + t_ops:.1f} s",
            "sample_candidates": n_done, "sample_seconds": t_spent + t_ops * n_done / N_CAND}


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
    sw, _, _ = build_inputs()
    from oracle import sblm as osb

    A_true = osb.magnification(sw.truth[None, :], sw.t)[0]
    sigma = sw.sigma_frac * A_true
    flux = A_true + sigma * sw.z
    # the whole run takes about REFERENCE_SECONDS whatever --steps and --warmup are: each step
    # times as many single candidates as fit in its share; the operators are timed once
    # a step is a bounded sample of the workload: the chi^2 of as many candidates as fit in its
    # share of the time, plus the operators' share of one generation for those candidates (the
    # operators of a whole generation are timed once). ms_per_step is the time a sampled step
    # took; the time the whole 4096 x 2000 step would take is projected separately
    per_step = max(0.02, REFERENCE_SECONDS / max(1, args.steps + args.warmup))
    t_ops = oracle_operator_seconds()
    step_s, n_cand = [], []
    for k in range(args.warmup + args.steps):
        cb = cpu_baseline(sw, flux, sigma, per_step, chunk=1, t_ops=t_ops)
        if k >= args.warmup:
            step_s.append(cb["sample_seconds"])
            n_cand.append(cb["sample_candidates"])
    value = float(np.sum(n_cand)) * N_EP / float(np.sum(step_s))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(step_s)) * 1e3,
            "projected_ms_per_step": N_POPS * N_CAND * N_EP / value * 1e3,
            "step": f"bounded sample: {float(np.mean(n_cand)):.1f} candidates of one population x {N_EP} epochs per "
                    f"step (chi^2) + the operators' share; projected_ms_per_step extrapolates to the whole step "
                    f"({N_POPS} x {N_CAND} candidates)",
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "populations": N_POPS, "candidates": N_CAND,
                                            "epochs": N_EP, "magnifications_per_step": N_POPS * N_CAND * N_EP},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": cb["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp32", "fp64"])
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--populations", type=int, default=N_POPS,
                    help="populations of 4096 candidates per step (32: the benchmark's workload; fewer for "
                         "profiling a smaller case of the same launch shape)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-fits", dest="fits", action="store_false", help="skip the fits/s measurement")
    ap.add_argument("--time-budget", type=float, default=1320.0,
                    help="seconds from the start within which the optional fit workloads must finish; a workload "
                         "that would not fit is reported as skipped")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="skip the end-to-end and other-precision measurements (profiling runs)")
    args = ap.parse_args()
    set_populations(args.populations)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
