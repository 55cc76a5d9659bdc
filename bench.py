#!/usr/bin/env python3
"""Throughput of the fused MHD stage on GB300: cell-updates/s.

One "step" is one full time step (two fused stages: ghost fill, primitive
recovery, limited reconstruction, Rusanov fluxes, Powell/B0 sources,
conservative update, CFL reduction) over every block of the workload.  A
cell-update is one cell advanced by one full step.

Default workload: 64 independent periodic block-adaptive grids of uneven size
(64..4096 blocks of 8^3 cells, log-uniform, seed 20250112) with smooth random
states, the mixed-precision form (FP32 reconstruction/fluxes/sources, FP64
pressure recovery and accumulation), one persistent launch per stage captured
in a CUDA graph with autotuned blocks per CTA.  The state (about 2 GB) is far
larger than L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--precision mixed|fp64] [--workload batched|blast|magnetosphere]

Prints one JSON line (rank 0).  Under torchrun each rank runs its own batch of
64 grids (seed offset by rank): weak scaling, no data-path collective.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

from paper_2501_06717_gb300 import workloads as W  # noqa: E402

METRIC = "cell-updates/s/GB300"
UNIT = "cell-updates/s"
BYTES_PER_CELL_UPDATE = 320  # FP64 state: stage 1 reads U^n, writes U*; stage 2 reads U*, U^n, writes U^{n+1}
# FP64 form: executed FP64 flops per cell-update (DADD + DMUL + 2 DFMA, both
# stages: 1,539 + 1,865), ncu counters of k_stage<0,...> on the first 8 grids
# of the batched workload (profiles/k_stage_fp64_batched8_ncu.md)
FP64_FLOPS_PER_CELL_UPDATE = 3404

# DRAM traffic of one k_stage launch per cell, from the ncu capture summarised
# in profiles/ (None until a capture of the current kernel source exists).
NCU_TRAFFIC = {
    # precision: (DRAM bytes per cell per launch, mean of the two stages, sha256 of the stage
    # kernel's sources -- bats_stage_kernel.h then bats_stage.cu -- at capture)
    "mixed": (127.6, "f9386682d83b66e714729f51ec395c92dfaf91250e1201ca309786ecc2cfb42b"),
}


def _peaks():
    p = os.path.join(HERE, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _bf16_peak():
    p = os.path.join(HERE, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["bf16_tflops"]), "measured (burst)"
    return 1900.0, "fallback"


def _kernel_sha():
    h = hashlib.sha256()
    for name in ("bats_stage_kernel.h", "bats_stage.cu"):
        with open(os.path.join(HERE, "paper_2501_06717_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def make_workload(name, rank=0, processes=None, grids=64):
    if name == "batched":
        probs = W.batched_grids(seed=20250112 + rank, processes=processes, first=grids)
        return probs, "%d independent periodic block-adaptive grids, 64-4096 blocks of 8^3 cells " \
            "(log-uniform, seed %d), smooth Fourier states" % (len(probs), 20250112 + rank)
    if name == "blast":
        return [W.blast()], "spherical MHD blast, 4^3 roots on [-1,1]^3 refined inside r<0.4 (120 blocks)"
    if name == "magnetosphere":
        return [W.magnetosphere()], "magnetosphere-like grid, 5 levels, dipole B0, body r=2.5 (3872 blocks)"
    raise ValueError(name)


def reduce_over_ranks(ms, cells, device):
    """Max of the timed-region durations and sum of the cells over all ranks
    (each rank advances its own batch: weak scaling, no data-path collective)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(cells)], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), float(c.item())


# --------------------------------------------------------------------------
# CPU oracle timing (test infrastructure; the baseline, not the target)


def oracle_sample(problems, seconds):
    """Run the oracle one step per grid over the workload's grids in order
    until `seconds` of CPU work; returns (cells, elapsed, grids used)."""
    from oracle import oracle as O
    O.build()
    cells = 0
    t0 = time.perf_counter()
    used = 0
    for p in problems:
        O.run(p, p.U0, 1, cfl=p.cfl)
        cells += p.ncells
        used += 1
        if time.perf_counter() - t0 >= seconds:
            break
    return cells, time.perf_counter() - t0, used


def cpu_baseline(problems, seconds):
    """The oracle with OpenMP over blocks on all host cores, and (a quarter of
    the time) on one core."""
    from oracle import oracle as O
    cells, el, used = oracle_sample(problems, seconds)
    cores = O.num_threads()
    O.set_threads(1)
    c1, e1, u1 = oracle_sample(problems, seconds / 4)
    O.set_threads(cores)
    return {"value": cells / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d of %d grids (%d cells), 1 step each, FP64 C oracle with OpenMP over blocks, %.1f s"
                      % (used, len(problems), cells, el),
            "single_core_value": c1 / e1,
            "single_core_sample": "%d grids (%d cells), 1 step each, %.1f s" % (u1, c1, e1)}


def run_reference(args, rank, world):
    """The oracle timed as the reference arm on the same workload, each step a
    bounded sample (the first grids of the workload)."""
    if rank != 0:
        return 0
    from oracle import oracle as O
    problems, desc = make_workload(args.workload, 0, processes=min(16, os.cpu_count() or 1), grids=args.grids)
    O.build()
    # size the sample for about 2.5 s per step
    t0 = time.perf_counter()
    O.run(problems[0], problems[0].U0, 1, cfl=problems[0].cfl)
    rate = problems[0].ncells / max(time.perf_counter() - t0, 1e-6)
    budget = rate * 2.5
    sample, cells = [], 0
    for p in problems:
        sample.append(p)
        cells += p.ncells
        if cells >= budget:
            break
    states = [p.U0.copy() for p in sample]
    for _ in range(args.warmup):
        for i, p in enumerate(sample):
            states[i], _, _ = O.run(p, states[i], 1, cfl=p.cfl)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for i, p in enumerate(sample):
            states[i], _, _ = O.run(p, states[i], 1, cfl=p.cfl)
        times.append(time.perf_counter() - t0)
    el = sum(times)
    value = cells * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": desc, "sample_grids": len(sample), "sample_cells": cells},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "sample": "first %d grids (%d cells) of the workload per step" % (len(sample), cells)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# Learned form: train on solver-made pairs, then time and score it


def learned_form_summary(stream, steps=32):
    """Blast at 1x (120 blocks) with the trained network against the plain
    scheme at 1x and 2x (960 blocks), fixed dt, FP64 and mixed forms; times
    from CUDA events around graph replays of `steps` coarse steps (2 * steps
    fine).  Errors are against the plain 2x run of the same precision,
    restricted to 1x, and (FP64) against a plain 4x run restricted to 1x, which
    also scores the plain 2x run."""
    import torch
    from paper_2501_06717_gb300 import bats, learn
    t0 = time.perf_counter()
    X, Y = learn.make_pairs(variants=list(range(101, 117)), snapshots=(4, 12, 20), keep=0.3)
    t_pairs = time.perf_counter() - t0
    t0 = time.perf_counter()
    P, hist = learn.train(X, Y, epochs=20, lr=2e-3)
    t_train = time.perf_counter() - t0
    e_plain, e_learn = learn.evaluate(P, nsteps=16)
    e_plain_m, e_learn_m = learn.evaluate(P, nsteps=16, precision=bats.BATS_MIXED)
    e4 = learn.evaluate_4x(P, nsteps=16)
    # the correction in the last stage of each step only (where its training
    # target is defined): the form timed below
    e4_last = learn.evaluate_4x(P, nsteps=16, last_only=1)
    coarse, fine = W.blast(), W.blast(resolution=2)
    coarse_last = W.Problem(**{**coarse.__dict__, "learned_last_only": 1})

    def timed(prob, params, nsteps, dt, precision):
        with bats.Solver(prob, precision=precision, stream=stream, persistent=1, use_graph=1) as s:
            if params is not None:
                s.set_mlp(params)
            s.set_state(0, prob.U0)
            s.step_dt(nsteps, dt)   # capture
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step_dt(nsteps, dt)
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / steps

    with bats.Solver(coarse) as s:
        s.set_state(0, coarse.U0)
        dtc = 0.5 * s.dt(0, 0.8)
    ms = {}
    for name, prec in (("fp64", bats.BATS_FP64), ("mixed", bats.BATS_MIXED)):
        ms[name] = {"learned_1x": timed(coarse_last, P, steps, dtc, prec),
                    "learned_1x_both_stages": timed(coarse, P, steps, dtc, prec),
                    "plain_1x": timed(coarse, None, steps, dtc, prec),
                    "plain_2x_two_fine_steps": timed(fine, None, 2 * steps, 0.5 * dtc, prec)}
    # the same network on a GPU-filling grid: the blast on 16^3 roots (6,056
    # blocks at 1x, 48,448 at 2x); timing only (the network was trained on the
    # 4^3-root blast; its inputs are scale-free)
    big1 = W.blast(roots_per_axis=16)
    big2 = W.blast(roots_per_axis=16, resolution=2)
    big1_last = W.Problem(**{**big1.__dict__, "learned_last_only": 1})
    with bats.Solver(big1) as s:
        s.set_state(0, big1.U0)
        dtb = 0.5 * s.dt(0, 0.8)
    nb = max(4, steps // 4)
    big = {"blocks_1x": big1.nb, "blocks_2x": big2.nb}
    for name, prec in (("fp64", bats.BATS_FP64), ("mixed", bats.BATS_MIXED)):
        r = {"learned_1x": timed(big1_last, P, nb, dtb, prec) * steps / nb,
             "learned_1x_both_stages": timed(big1, P, nb, dtb, prec) * steps / nb,
             "plain_1x": timed(big1, None, nb, dtb, prec) * steps / nb,
             "plain_2x_two_fine_steps": timed(big2, None, 2 * nb, 0.5 * dtb, prec) * steps / nb}
        big[name] = {"ms_per_coarse_step": r,
                     "cell_updates_per_s": {"learned_1x": big1.ncells / (r["learned_1x"] * 1e-3),
                                            "plain_1x": big1.ncells / (r["plain_1x"] * 1e-3),
                                            "plain_2x": 2 * big2.ncells / (r["plain_2x_two_fine_steps"] * 1e-3)}}
    return {"workload": "spherical blast: 120 blocks (1x) with the trained network vs plain 1x and plain 2x "
                        "(960 blocks), fixed dt, CUDA graph",
            "pairs": int(X.shape[0]), "pairs_s": t_pairs, "train_s": t_train, "train_epochs": 20, "train_batch": 8192, "loss_first_last_epoch": [hist[0], hist[-1]],
            "error_vs_restricted_2x": {"plain_1x": e_plain, "learned_1x": e_learn,
                                       "plain_1x_mixed": e_plain_m, "learned_1x_mixed": e_learn_m},
            "error_vs_restricted_4x_fp64": {**e4, "learned_1x_both_stages": e4["learned_1x"],
                                            "learned_1x": e4_last["learned_1x"]},
            "learned_form": "correction in the last stage of each step (learned_last_only)",
            "ms_per_coarse_step": ms,
            "gpu_filling_blast_16cube_roots": big,
            "cell_updates_per_s_learned_1x": {k: coarse.ncells / (v["learned_1x"] * 1e-3) for k, v in ms.items()}}


# --------------------------------------------------------------------------
# The network alone on the tensor cores

MLP_FLOPS_PER_ROW = 2 * (40 * 64 + 64 * 64 + 64 * 8)   # 14,336 algorithmic
MLP_BYTES_PER_ROW = 48 * 2 + 8 * 4                      # BF16 inputs (padded to 48) + FP32 outputs


def mlp_inference_summary(stream, rows=2_000_000, reps=20):
    """k_mlp_infer over `rows` face rows of N(0, 1) BF16 inputs (192 MB of
    inputs, larger than L2) with a seeded network, timed with CUDA events on
    the handle's stream over `reps` back-to-back launches."""
    import torch
    from paper_2501_06717_gb300 import bats
    g = torch.Generator(device="cuda").manual_seed(5)
    Xh = torch.zeros(rows, 48, dtype=torch.bfloat16, device="cuda")
    Xh[:, :40] = torch.randn(rows, 40, device="cuda", generator=g).to(torch.bfloat16)
    Xb = Xh.view(torch.int32)
    Y = torch.empty(rows, 8, device="cuda")
    P = (0.3 * np.random.default_rng(6).normal(size=bats.BATS_MLP_NPARAM)).astype(np.float32)
    m = bats.Mlp(P, stream=stream)
    torch.cuda.synchronize()
    for _ in range(3):
        m.forward_bf16(Xb, Y)
    m.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        m.forward_bf16(Xb, Y)
    e1.record(stream)
    m.sync()
    ms = e0.elapsed_time(e1) / reps
    m.close()
    peak, how = _bf16_peak()
    hbm, hbm_how = _peaks()
    tf = rows * MLP_FLOPS_PER_ROW / (ms * 1e-3) / 1e12
    gbs = rows * MLP_BYTES_PER_ROW / (ms * 1e-3) / 1e9
    return {"kernel": "k_mlp_infer", "rows": rows, "ms_per_launch": ms, "rows_per_s": rows / (ms * 1e-3),
            "flops_per_row": MLP_FLOPS_PER_ROW, "tflops": tf, "bf16_peak_tflops": peak, "peak_kind": how,
            "frac_bf16_peak": tf / peak, "bytes_per_row": MLP_BYTES_PER_ROW, "gbs": gbs,
            "frac_hbm": gbs / hbm, "hbm_peak_kind": hbm_how, "inputs": "larger than L2"}


# --------------------------------------------------------------------------
# The other paper-shaped grids (one grid each)


def other_workloads(stream, steps=20, fp64_steps=4):
    """Mixed and FP64 throughput on the blast at 16^3 roots, the magnetosphere
    stand-in and the Table 2 fast-wave grid at m = 12 (with the Rusanov and
    with the HLL flux), each one grid in one persistent launch per stage
    replayed from a CUDA graph."""
    import torch
    from paper_2501_06717_gb300 import bats

    def with_hll(prob):
        prob.flux = W.FLUX_HLL
        return prob

    out = {}
    for name, make in (("blast_16cube_roots", lambda: W.blast(roots_per_axis=16)),
                       ("magnetosphere", W.magnetosphere),
                       ("fast_wave_table2_m12", lambda: W.fast_wave(m=12)),
                       ("fast_wave_table2_m12_hll", lambda: with_hll(W.fast_wave(m=12)))):
        prob = make()
        row = {"blocks": prob.nb, "cells": prob.ncells}
        for pname, prec, n in (("mixed", bats.BATS_MIXED, steps), ("fp64", bats.BATS_FP64, fp64_steps)):
            with bats.Solver(prob, precision=prec, stream=stream, persistent=1, use_graph=1) as s:
                s.set_state(0, prob.U0)
                s.step(n, prob.cfl)   # captures the n-step graph
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s.step(n, prob.cfl)
                e1.record(stream)
                torch.cuda.synchronize()
                row[pname] = prob.ncells * n / (e0.elapsed_time(e1) * 1e-3)
        del prob
        out[name] = row
    # Section 5.1's one-GPU run: the Table 2 fast-wave grid at m = 6 (960
    # blocks of 8^3 here; 10^3 in the paper) with the Linde flux, 500 steps at
    # CFL 0.8, one CUDA graph of all 500 steps per precision
    prob = W.fast_wave(m=6)
    prob.flux = W.FLUX_LINDE
    row = {"blocks": prob.nb, "cells": prob.ncells, "steps": 500, "flux": "linde",
           "paper_table3_one_gpu_total_s": {"A100": 5.76, "V100": 7.68},
           "paper_cells": prob.nb * 1000}
    for pname, prec in (("mixed", bats.BATS_MIXED), ("fp64", bats.BATS_FP64)):
        with bats.Solver(prob, precision=prec, stream=stream, persistent=1, use_graph=1) as s:
            s.set_state(0, prob.U0)
            s.step(500, prob.cfl)   # captures the 500-step graph
            s.set_state(0, prob.U0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step(500, prob.cfl)
            e1.record(stream)
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) * 1e-3
            row[pname] = {"total_s": sec, "cell_updates_per_s": prob.ncells * 500 / sec}
    out["fast_wave_table2_m6_linde_500_steps"] = row
    return out


# --------------------------------------------------------------------------
# Clocks during the timed region


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "50",
                 "-i", str(gpu_index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# GPU arm


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--workload", default="batched", choices=["batched", "blast", "magnetosphere"])
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--grids", type=int, default=64, help="first N grids of the batched workload")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-form summary")
    ap.add_argument("--learned-only", action="store_true", help="only the learned-form summary (profiling)")
    ap.add_argument("--no-others", action="store_true", help="skip the other paper-shaped grids")
    ap.add_argument("--mlp-only", action="store_true", help="only the standalone network inference (profiling)")
    ap.add_argument("--others-only", action="store_true", help="only the other paper-shaped grids")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and "RANK" not in os.environ:
        raise SystemExit("--gpus > 1 needs torchrun (one process per GPU)")
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.others_only:
        import torch
        torch.cuda.set_device(local)
        print(json.dumps({"other_workloads_cell_updates_per_s": other_workloads(torch.cuda.Stream())}), flush=True)
        return 0
    if args.mlp_only:
        import torch
        torch.cuda.set_device(local)
        print(json.dumps({"mlp_inference": mlp_inference_summary(torch.cuda.Stream())}), flush=True)
        return 0
    if args.learned_only:
        import torch
        torch.cuda.set_device(local)
        print(json.dumps({"learned_form": learned_form_summary(torch.cuda.Stream())}), flush=True)
        return 0

    # inputs and the CPU baseline before any CUDA call (spawned pool only)
    problems, desc = make_workload(args.workload, rank, processes=min(16, os.cpu_count() or 1), grids=args.grids)
    cpu = cpu_baseline(problems, args.cpu_seconds) if (rank == 0 and world == 1 and args.cpu_seconds > 0) else None

    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2501_06717_gb300 import autotune, bats

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    prec = bats.BATS_MIXED if args.precision == "mixed" else bats.BATS_FP64
    stream = torch.cuda.Stream()
    cells = sum(p.ncells for p in problems)
    cfl = problems[0].cfl
    solver = bats.Solver(problems, precision=prec, stream=stream)
    solver.set_states()

    # warm-up: autotune the launch form, then W steps, then build the graph
    tune = None
    if not args.no_autotune:
        tune = autotune.autotune(solver, cfl, steps=2)
    else:
        solver.set_launch(1, 1, 0, 1)
    for _ in range(args.warmup):
        solver.step(1, cfl)
    solver.step(args.steps, cfl)  # captures the K-step graph

    torch.cuda.synchronize()
    barrier()
    clocks = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ
                          else os.environ["CUDA_VISIBLE_DEVICES"].split(",")[local])
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        ev0.record(stream)
        solver.step(args.steps, cfl)
        ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    launches = solver.launch_count()
    # mean stage-kernel launch duration in the timed region itself: the
    # replayed graph's own event nodes bracket each step's two stage launches
    # (ghost pre-pass included) on the handle's stream
    stage_ms = solver.timings()[bats.BATS_PHASE_STAGE]
    stage_total_ms = solver.timings()[bats.BATS_PHASE_TOTAL]
    if world > 1:
        ms, total_cells = reduce_over_ranks(ms, cells, "cuda")
    else:
        total_cells = cells
    value = total_cells * args.steps / (ms * 1e-3)

    # roofline of the dominant kernel (k_stage): algorithmic bytes per launch
    # (160 B per cell on average over the two stages) / mean launch duration
    nlaunch = 2 * args.steps
    per_launch_ms = stage_ms / nlaunch
    alg_bytes = BYTES_PER_CELL_UPDATE / 2 * cells
    achieved = alg_bytes / (per_launch_ms * 1e-3) / 1e9
    peak, peak_kind = _peaks()
    tr = NCU_TRAFFIC.get(args.precision)
    traffic = tr[0] * cells if (tr and tr[1] == _kernel_sha()) else None

    # end to end through the public API with host buffers: per step, every
    # grid's state goes in from pinned host memory and comes back out (one
    # transfer each way for the whole batch)
    host = None
    if args.e2e_steps:
        host = torch.from_numpy(np.concatenate([np.ascontiguousarray(p.U0).reshape(-1) for p in problems])).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        bats.bats_set_states(solver.h, host)
        solver.step(1, cfl)
        bats.bats_get_states(solver.h, host)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    state_bytes = cells * 8 * 8
    e2e = {"value": cells * args.e2e_steps / e2e_s * (total_cells / cells) if args.e2e_steps else None, "unit": UNIT,
           "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes}

    # the plain FP64 path on the same workload, for the mixed-vs-FP64 comparison
    fp64 = None
    fp64_roofline = None
    if prec == bats.BATS_MIXED and args.fp64_steps > 0:
        solver.close()
        s64 = bats.Solver(problems, precision=bats.BATS_FP64, stream=stream, persistent=1, blocks_per_cta=1)
        s64.set_states()
        s64.step(2, cfl)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s64.step(args.fp64_steps, cfl)
        e1.record(stream)
        torch.cuda.synchronize()
        fp64 = cells * args.fp64_steps / (e0.elapsed_time(e1) * 1e-3)
        s64.close()
        # its roofline: the FP64 pipe.  Executed FP64 flops per cell-update
        # (DADD + DMUL + 2 DFMA, both stages) from the ncu counters of the
        # FP64 stage kernel; the peak is this GPU's FP64 FMA rate, measured now
        peak64 = bats.bats_fp64_fma_rate(stream)
        achieved64 = FP64_FLOPS_PER_CELL_UPDATE * fp64 / 1e9
        fp64_roofline = {"bound": "fp64", "achieved": achieved64, "peak": peak64, "unit": "GFLOP/s",
                         "frac": achieved64 / peak64 if peak64 > 0 else None,
                         "flops_per_cell_update": FP64_FLOPS_PER_CELL_UPDATE,
                         "peak_source": "measured (bats_fp64_fma_rate: independent FMA chains)"}

    learned = None
    if rank == 0 and world == 1 and not args.no_learned and args.workload == "batched":
        learned = learned_form_summary(stream)
        learned["mlp_inference_2M_rows"] = mlp_inference_summary(stream)
    others = None
    if rank == 0 and world == 1 and not args.no_others and args.workload == "batched":
        others = other_workloads(stream)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if prec == bats.BATS_MIXED else "f64", "data": "synthetic",
            "config": {"workload": desc, "blocks": sum(p.nb for p in problems), "cells_per_gpu": cells,
                       "precision": args.precision,
                       "launch": {"persistent_blocks_per_cta_ctas_per_sm": list(tune[0][:3]) if tune else [1, 1, 0],
                                  "staging": (None if not tune or tune[0][3] is None
                                              else ("tma" if tune[0][3] else "gather")),
                                  "cuda_graph": True},
                       "l2": "inputs larger than L2 (state %.2f GB per GPU, L2 129 MB); no flush" %
                             (2 * state_bytes / 1e9),
                       "cfl": cfl},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": ("k_stage<true> with its ghost pre-pass k_amr_ghosts" if prec == bats.BATS_MIXED
                                    else "k_stage<false>"),
                         "peak_source": peak_kind, "bytes_per_launch": alg_bytes,
                         "mean_launch_ms": per_launch_ms},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
            "fp64_value": fp64,
            "fp64_roofline": fp64_roofline,
            "learned_form": learned,
            "other_workloads_cell_updates_per_s": others,
            "stage_share": stage_ms / stage_total_ms if stage_total_ms > 0 else None,
        }
        if tune:
            line["autotune_ms_per_stage"] = {
                "%d/%d/%d%s" % (c[:3] + ("" if c[3] is None else "/" + ("tma" if c[3] else "gather"),)): m
                for c, m in tune[1]}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
