#!/usr/bin/env python3
"""Benchmark of the evaluate-and-stamp hot path (one JSON line on stdout).

A step is one Newton-iteration eval_stamp of the whole workload: every MOSFET evaluated (currents,
charges, conductances) and stamped into A and b. Default workload: random CMOS logic of 277,778
INV/NAND2/NOR2 gates (~1.0M MOSFETs, the million-device netlist of the throughput bar), node
voltages U[0, 1] V, sizes W ~ U[0.5, 5] um, L ~ U[0.1, 1] um, all from the fixed seed. Inputs are
resident in HBM; a 256 MiB buffer is written between timed steps so every step starts with a
cold L2. The SRAM (256 x 256 6T), the backward, the transient stamp, the batch of 4,096 circuits
and the 64-bit adder study are reported under "extras".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload ...]

N > 1 (under torchrun): rank r evaluates its own netlist (the same generator, seed + r) -- or,
with --workload batch, its round-robin share of the 4,096 circuits (circuits r, r + N, ...);
no collective on the data path (weak scaling); rank 0 prints the aggregate. ``--impl
reference`` times the serial CPU oracle on the host cores on the same workload and metric.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MOSFET eval+stamp/s per NR iter (FP64, 1xGB300)"
UNIT = "device evals+stamps/s"
# Per-device work of the dominant kernel, per workload and kernel, from ncu's counters of one
# launch: FP64 flop = 2 DFMA + DADD + DMUL thread instructions per device, and DRAM bytes read +
# written per device (summaries and commands in profiles/). Kernels: "eval_cost" = k_eval_ranges
# (atomic schedule, cost order), "eval_layout" = k_eval (atomic, layout order), "pipe" =
# k_color_pipe (pipelined colour schedule, evaluation and stamp in one kernel). The counts hold
# for the kernel sources they were taken on (COUNTED_SOURCES_SHA16, a hash of the files in
# KERNEL_SOURCES): once those change, the bench flags the figures as stale and reports no
# traffic until they are counted again.
KERNEL_SOURCES = ("eec_model.cuh", "eec_fastmath.cuh", "eec_tables.h", "eec_internal.h",
                  "eec_kernels.cu")
COUNTED_SOURCES_SHA16 = "e458d79fa8bce390"
COUNTS = {    # (workload, kernel) -> (FP64 flop per device, DRAM bytes per device)
    ("logic1m", "eval_cost"): (255.46, 292.15),
    ("batch", "eval_cost"): (234.78, 376.16),
    ("sram", "eval_cost"): (265.86, 185.02),
    ("logic1m", "pipe"): (258.24, 284.98),
}
# GB300: 152 SMs x 2 FP64 FMA per clock per SM x 2 flop x 2070 MHz maximum SM clock.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12


def kernel_sources_sha16():
    """Hash of the evaluate kernels' sources (the files the counted figures depend on)."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2604_03079_gb300", "csrc", f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["sram", "logic", "logic1m", "logic120k", "batch", "chain"],
                    default="logic1m",
                    help="logic120k: 120,000 gates (~430k FETs), a profiling case whose inputs "
                         "still exceed L2")
    ap.add_argument("--variant", default="auto")
    ap.add_argument("--eval-order", choices=["auto", "cost", "layout"], default="auto",
                    help="evaluation launch order of the order-free schedules (auto: the "
                         "autotuner's choice; with --quick, cost)")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--quick", action="store_true",
                    help="timed steps only (no autotune, e2e, extras, probes, baseline): for ncu")
    ap.add_argument("--bwd-steps", type=int, default=0,
                    help="with --quick: also run the backward this many times (for ncu)")
    ap.add_argument("--newton", action="store_true",
                    help="only run the GPU Newton-loop study (NEXT-2) and print it as JSON")
    ap.add_argument("--tran-steps", type=int, default=0,
                    help="with --quick: also run the trapezoidal transient stamp this many times "
                         "(for ncu)")
    return ap.parse_args()


def workload(name, world=1, rank=0):
    """(netlist or None, circuits or None, description) of a workload; with world > 1 the share
    of this rank (its own netlist, seed + rank; for the batch its round-robin circuits)."""
    import netgen
    seed = netgen.DEFAULT_SEED + rank
    if name == "batch":
        nets = netgen.batch_circuits(4096)
        if world > 1:
            nets = netgen.shard(nets, world, rank)
        return None, nets, "batch_4096_circuits_merged"
    if name == "sram":
        return netgen.sram(256, 256, seed), None, "sram_256x256_6T (393216 MOSFETs)"
    if name == "logic":
        return netgen.random_logic(200_000, seed), None, "random_logic_200k_gates"
    if name == "logic1m":
        return (netgen.random_logic(277_778, seed), None,
                "random_logic_277778_gates (~1M MOSFETs)")
    if name == "logic120k":
        return netgen.random_logic(120_000, seed), None, "random_logic_120000_gates"
    return netgen.inverter_chain(64, seed), None, "inverter_chain_64"


class Clocks:
    """nvidia-smi sampling during the timed region (SM clock, reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.3)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def reduce_max(value, device=None):
    """Max of a per-rank number over the default process group (identity on one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(n_dev_all_ranks, ms_per_step):
    """Whole-job throughput: the devices of every rank per step, over the slowest rank's step
    time (weak scaling: each rank's share is fixed as the rank count grows)."""
    return n_dev_all_ranks / (ms_per_step * 1e-3)


def sum_over_ranks(value, device=None):
    """Sum of a per-rank number over the default process group (identity on one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def parity_vs_oracle(o, x, A, b, q, tol=1e-12):
    """Full-size parity of one GPU step (host copies of A, b, q) against the oracle, untimed:
    per entry the cancellation-aware error |gpu - oracle| / max(|oracle|, S_e), S_e the sum of
    |contributions| into the entry (the tests' criterion, at most tol), beside the plain relative
    error |gpu - oracle| / |oracle| over the entries where the oracle is not zero; charges
    relative to each device's largest terminal charge."""
    r = o.eval_stamp(x, want_q=True, want_scale=True)
    rec = {"tol": tol}
    ok = True
    for k, got, ref, sc in (("A", A, r["A"], r["A_scale"]), ("b", b, r["b"], r["b_scale"])):
        den = np.maximum(np.abs(ref), sc)
        den = np.where(den == 0, 1.0, den)
        err = np.abs(got - ref) / den
        nz = ref != 0
        plain = np.abs(got[nz] - ref[nz]) / np.abs(ref[nz])
        rec[k] = {"entries": int(ref.size), "max_err": float(err.max(initial=0.0)),
                  "max_plain": float(plain.max(initial=0.0)),
                  "p99_plain": float(np.quantile(plain, 0.99)) if plain.size else 0.0,
                  "median_plain": float(np.median(plain)) if plain.size else 0.0}
        ok = ok and rec[k]["max_err"] <= tol
    if r["q"].size:
        qg = q.reshape(4, -1)
        scale = np.maximum(np.abs(r["q"]).max(axis=0, keepdims=True), 1e-300)
        rec["q"] = {"max_err": float((np.abs(qg - r["q"]) / scale).max())}
    rec["pass"] = bool(ok)
    return rec


def cpu_baseline(net, x, budget_s=10.0, gpu_step=None):
    """The oracle as it stands, single-threaded, on the host: full workload, repeated. With
    gpu_step = (A, b, q) from the GPU at the same x, also the full-size parity record (one
    untimed oracle call with the error scales)."""
    import netgen
    import oracle
    o = oracle.Oracle(net, netgen.default_cards())
    parity = parity_vs_oracle(o, x, *gpu_step) if gpu_step is not None else None
    reps, t0 = 0, time.perf_counter()
    while True:
        o.eval_stamp(x, want_q=True)
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or (reps >= 1 and el * (reps + 1) / reps > 3 * budget_s):
            break
    out = {"value": net.n_dev * reps / el, "unit": UNIT, "cores": 1,
           "host_cores_available": len(os.sched_getaffinity(0)), "kind": "oracle",
           "sample": f"whole workload ({net.n_dev} devices) x {reps} eval_stamp calls, "
                     f"{el:.1f} s, 1 thread"}
    return out, parity


def _merged(net, nets):
    import netgen
    return net if net is not None else netgen.concat(nets)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import netgen
    import oracle
    net, nets, wname = workload(args.workload)
    net = _merged(net, nets)
    x = netgen.random_x(net)
    o = oracle.Oracle(net, netgen.default_cards())
    # bounded steps: the oracle takes one to two seconds per step on the default workload
    steps = max(1, min(args.steps, 20))
    warm = max(0, min(args.warmup, 2))
    for _ in range(warm):
        o.eval_stamp(x, want_q=True)
    t0 = time.perf_counter()
    for _ in range(steps):
        o.eval_stamp(x, want_q=True)
    el = time.perf_counter() - t0
    v = net.n_dev * steps / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 0,
            "steps": steps, "warmup": warm, "ms_per_step": 1e3 * el / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wname, "sample": "whole workload"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"whole workload ({net.n_dev} devices) x {steps} steps"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def make_context(eec, net, nets, cards):
    if nets is not None:
        return eec.Circuit(None, cards, color=True, batch=nets)
    return eec.Circuit(net, cards, color=True)


def timed_steps(eec, circ, xt, A, b, q, steps, warmup, flush, stream, world):
    """Warm-up, then `steps` steps bracketed by barrier + synchronize, each after an L2 flush,
    timed with CUDA events on the launching stream; returns (per-step ms, library kernels)."""
    import torch
    import torch.distributed as dist
    for _ in range(warmup):
        circ.eval_stamp(xt, A, b, q)
    torch.cuda.synchronize()
    assert circ.status() == 0
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    eec.eec_profile_read(circ.ctx)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(steps):
        flush.zero_()
        ev[i][0].record(stream)
        circ.eval_stamp(xt, A, b, q)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    prof = eec.eec_profile_read(circ.ctx)
    return [a.elapsed_time(bb) for a, bb in ev], prof["kernels"]


def phase_split(eec, circ, xt, A, b, q, steps, flush):
    """init / evaluate / stamp per step from CUDA events around the phases (a second pass: an
    event between the initialisation and the evaluation keeps them from overlapping)."""
    eec.eec_profile_enable(circ.ctx, True)
    eec.eec_profile_read(circ.ctx)
    for _ in range(steps):
        flush.zero_()
        circ.eval_stamp(xt, A, b, q)
    prof = eec.eec_profile_read(circ.ctx)
    eec.eec_profile_enable(circ.ctx, False)
    n = max(prof["calls"], 1)
    return {"init": prof["ms_init"] / n, "eval": prof["ms_eval"] / n, "stamp": prof["ms_stamp"] / n}


def dominant_kernel(eec, circ, variant):
    """(key into COUNTS, kernel name) of the kernel that dominates a step of this schedule."""
    if variant == eec.EEC_VARIANT_COLOR_PIPELINED:
        return "pipe", "k_color_pipe (evaluate and stamp)"
    if variant == eec.EEC_VARIANT_ATOMIC:
        if eec.eec_get_tuning(circ.ctx)[2]:
            return "eval_cost", "k_eval_ranges (evaluate, cost order)"
        return "eval_layout", "k_eval (evaluate, layout order)"
    return None, f"evaluate kernel of {eec.VARIANT_NAMES[variant]}"


def roofline(eec, circ, variant, wkey, n_dev, kernel_ms):
    key, kname = dominant_kernel(eec, circ, variant)
    sha = kernel_sources_sha16()
    fresh = COUNTED_SOURCES_SHA16 is not None and sha == COUNTED_SOURCES_SHA16
    cnt = COUNTS.get((wkey, key)) if key else None
    if cnt and not fresh:
        sys.stderr.write("bench: the counted FP64/DRAM figures were taken on other kernel "
                         f"sources ({COUNTED_SOURCES_SHA16} != {sha}); recount them with ncu\n")
    flop = cnt[0] if cnt else None
    ach = flop * n_dev / (kernel_ms * 1e-3) / 1e12 if (flop and kernel_ms > 0) else None
    return {"bound": "alu", "kernel": kname, "achieved": ach, "peak": FP64_PEAK_TFLOPS,
            "unit": "TFLOP/s", "frac": (ach / FP64_PEAK_TFLOPS) if ach else None,
            "traffic": (cnt[1] * n_dev) if (cnt and fresh) else None,
            "flop_per_device": flop, "counts_fresh": bool(cnt and fresh),
            "kernel_sources_sha16": sha, "kernel_ms": kernel_ms,
            "peak_source": "152 SM x 2 DFMA/clk x 2 flop x 2070 MHz (maximum SM clock; nominal "
                           "1.25 TFLOP/s FP64); the library's DFMA probe is fp64_probe_tflops"}


def run_ours(args):
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    from paper_2604_03079_gb300 import build as _build
    _build.build()
    import netgen
    import paper_2604_03079_gb300 as eec

    dev = torch.device("cuda", torch.cuda.current_device())
    net, nets, wname = workload(args.workload, world, rank)
    mnet = _merged(net, nets)
    x = netgen.random_x(mnet)
    cards = netgen.default_cards()
    circ = make_context(eec, net, nets, cards)
    xt = torch.as_tensor(x, device=dev)
    A, b, q = circ.new_outputs(want_q=True)
    ms_variants = [] if args.quick else eec.eec_autotune(circ.ctx, xt, A, b, q, reps=5)
    if args.variant != "auto":
        eec.eec_set_variant(circ.ctx, int(args.variant))
    if args.eval_order != "auto":
        eec.eec_set_eval_order(circ.ctx, 1 if args.eval_order == "cost" else 0)
    variant = eec.eec_get_variant(circ.ctx)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    clocks = Clocks(torch.cuda.current_device()) if (rank == 0 and not args.quick) else None
    if clocks:
        clocks.start()
    step_ms, launches = timed_steps(eec, circ, xt, A, b, q, args.steps, args.warmup, flush,
                                    stream, world)
    clk = clocks.stop() if clocks else None
    total_ms = reduce_max(float(sum(step_ms)), dev)
    assert circ.status() == 0
    ms_per_step = total_ms / args.steps
    n_dev_all = sum_over_ranks(circ.n_dev, dev)
    value = aggregate_value(n_dev_all, ms_per_step)
    phases = phase_split(eec, circ, xt, A, b, q, args.steps, flush)

    if world > 1:
        sharding = ("round-robin share of the 4,096 circuits per rank (circuits r, r + N, ...)"
                    if nets is not None else "own netlist per rank (same generator, seed + rank)")
    else:
        sharding = "single GPU"
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step,
           "ms_per_step_median": statistics.median(step_ms), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded netlist generators, random-init node voltages)",
           "config": {"workload": wname, "n_dev": circ.n_dev, "n_dev_all_ranks": int(n_dev_all),
                      "n_unknowns": circ.n, "nnz": circ.nnz, "colors": circ.n_colors,
                      "variant": eec.VARIANT_NAMES[variant],
                      "block": (eec.eec_get_tuning(circ.ctx)[1] or
                                "library choice: 32 for launches under 19,456 devices, else 128"),
                      "eval_order": ("free source/body first" if eec.eec_get_tuning(circ.ctx)[2]
                                     else "layout order"),
                      "l2": "flushed (256 MiB write) before every timed step",
                      "parallelism": f"dp{world}: {sharding}" if world > 1 else sharding},
           "gpu_launches": launches,
           "phases_ms": phases}
    if clk:
        out["clocks"] = clk

    if rank == 0 and args.quick:
        if args.bwd_steps:
            rng = netgen.Rng(netgen.DEFAULT_SEED, 12)
            gA = torch.as_tensor(rng.normal(circ.nnz), device=dev)
            gb = torch.as_tensor(rng.normal(circ.n), device=dev)
            for _ in range(args.bwd_steps):
                circ.bwd(xt, gA, gb)
            torch.cuda.synchronize()
            assert circ.status() == 0
        if args.tran_steps:
            qprev = torch.empty_like(q)
            circ.eval_stamp(xt, A, b, qprev)
            ic, ip = torch.empty_like(q), torch.zeros_like(q)
            for _ in range(args.tran_steps):
                eec.eec_eval_stamp_tran(circ.ctx, xt, qprev, ip, 2e11, 1.0, A, b, q, ic)
            torch.cuda.synchronize()
            assert circ.status() == 0
        print(json.dumps(out))
    elif not args.quick:
        # the evaluate phase is the dominant kernel's time (the whole kernel under the
        # pipelined schedule, whose stamp runs inside it)
        out["roofline"] = roofline(eec, circ, variant, args.workload, circ.n_dev, phases["eval"])
        out["variants_ms"] = {eec.VARIANT_NAMES[i]: m for i, m in enumerate(ms_variants)}
        # end to end through the public API with host buffers (pinned): every step copies its
        # x in and its A, b, q out inside the timed region
        out["e2e"] = e2e(eec, circ, x, args, dev, world, n_dev_all)
        if rank == 0:
            out["fp64_probe_tflops"] = eec.eec_fp64_peak(4096, 8) / 1e12
            if world == 1 and not args.no_extras:
                out["extras"] = extras(eec, circ, mnet, x, xt, A, b, q, args, dev)
            if world == 1:
                # one more step of the timed schedule at the same x (the extras reuse A and b),
                # for the parity record
                circ.eval_stamp(xt, A, b, q)
                torch.cuda.synchronize()
                step = tuple(t.cpu().numpy() for t in (A, b, q))
                out["cpu_baseline"], out["parity"] = cpu_baseline(mnet, x, gpu_step=step)
                out["gpu_over_oracle"] = value / out["cpu_baseline"]["value"]
            print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()
    return 0


def e2e(eec, circ, x, args, dev, world, n_dev):
    """n_dev: the devices of all ranks (the whole job's work per step)."""
    import torch
    cs = torch.cuda.current_stream()
    ts_in, ts_out = torch.cuda.Stream(), torch.cuda.Stream()   # copies in / out overlap
    xh = torch.as_tensor(x).pin_memory()
    xd = [torch.empty(circ.n, dtype=torch.float64, device=dev) for _ in range(2)]
    outs = [circ.new_outputs(want_q=True) for _ in range(2)]
    hosts = [tuple(torch.empty(t.numel(), dtype=torch.float64).pin_memory() for t in o)
             for o in outs]
    ev = {k: [torch.cuda.Event() for _ in range(2)] for k in ("h2d", "eval", "d2h")}
    steps = max(10, min(args.steps, 400))

    # (a) the C-ABI call with host buffers, one call per step on one stream (serial)
    hA = torch.empty(circ.nnz, dtype=torch.float64).pin_memory()
    hb = torch.empty(circ.n, dtype=torch.float64).pin_memory()
    hq = torch.empty(4 * circ.n_dev, dtype=torch.float64).pin_memory()
    for _ in range(3):
        eec.eec_eval_stamp_host(circ.ctx, xh, hA, hb, hq, cs)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(cs)
    for _ in range(steps):
        eec.eec_eval_stamp_host(circ.ctx, xh, hA, hb, hq, cs)
    e1.record(cs)
    torch.cuda.synchronize()
    ms_host = e0.elapsed_time(e1) / steps

    # (b) device buffers with the copies pipelined by the caller
    def step(i):
        s = i & 1
        A, b, q = outs[s]
        with torch.cuda.stream(ts_in):
            if i >= 2:
                ts_in.wait_event(ev["eval"][s])   # x buffer s free again
            xd[s].copy_(xh, non_blocking=True)
            ev["h2d"][s].record(ts_in)
        cs.wait_event(ev["h2d"][s])
        if i >= 2:
            cs.wait_event(ev["d2h"][s])           # outputs of step i-2 are on the host
        eec.eec_eval_stamp(circ.ctx, xd[s], A, b, q, cs)
        ev["eval"][s].record(cs)
        with torch.cuda.stream(ts_out):
            ts_out.wait_event(ev["eval"][s])
            for hdst, dsrc in zip(hosts[s], (A, b, q)):
                hdst.copy_(dsrc, non_blocking=True)
            ev["d2h"][s].record(ts_out)

    for i in range(4):
        step(i)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(cs)
    for i in range(steps):
        step(i)
    cs.wait_stream(ts_out)
    e1.record(cs)
    torch.cuda.synchronize()
    ms_pipe = e0.elapsed_time(e1) / steps
    ms_host = reduce_max(ms_host, dev)     # the slowest rank (identity on one rank)
    ms_pipe = reduce_max(ms_pipe, dev)
    return {"value": n_dev / (ms_host * 1e-3), "unit": UNIT,
            "h2d_bytes_per_step": 8 * circ.n,
            "d2h_bytes_per_step": 8 * (circ.nnz + circ.n + 4 * circ.n_dev),
            "ms_per_step": ms_host,
            "how": "one eec_eval_stamp_host call per step, serial as in a Newton loop: x copied "
                   "in from page-locked memory, A, b and q copied out (q span by span while later "
                   "spans are evaluated)",
            "pipelined_device_buffers": {
                "value": n_dev / (ms_pipe * 1e-3), "ms_per_step": ms_pipe,
                "how": "eec_eval_stamp on device buffers, input and output copies on their own "
                       "streams, double-buffered across steps (independent evaluations)"}}


def hbm_peak_gbs():
    """(GB/s, source): the measured copy bandwidth of this GPU pool, else the fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json, STREAM-style copy)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback (6.8 TB/s, one earlier GB300 copy measurement)"


def newton_study(eec, dev, stream):
    """NEXT-2: the DC Newton loop closed on the GPU (evaluate and stamp, a sparse solve, damped
    update) from x = 0, per netlist and solver (0: cuSOLVER batched QR, analysis reused; 1:
    cuSOLVER QR after AMD; 2: the library's sparse LU, host analysis once, GPU refactorisation):
    iterations, time per iteration and the evaluate-and-stamp share of it (the paper: once
    evaluation is fast, the solve dominates). Bounded: at most 300 iterations per netlist and
    about a minute and a half in all."""
    import torch
    import netgen
    out = {}
    t_start = time.perf_counter()
    for nname, nn, solver in (("ripple_adder_64", netgen.ripple_adder(64), 2),
                              ("ripple_adder_64", netgen.ripple_adder(64), 0),
                              ("ripple_adder_64", netgen.ripple_adder(64), 1),
                              ("sram_32x32", netgen.sram(32, 32), 2),
                              ("sram_128x128", netgen.sram(128, 128), 2),
                              ("inverter_chain_1024", netgen.inverter_chain(1024), 2),
                              ("inverter_chain_1024", netgen.inverter_chain(1024), 1),
                              ("inverter_chain_4096", netgen.inverter_chain(4096), 2)):
        nname = f"{nname}_solver{solver}"
        if time.perf_counter() - t_start > 90:
            out[nname] = {"skipped": "time budget of the study used up"}
            continue
        c = eec.Circuit(nn, netgen.default_cards(), color=True)
        xd = torch.zeros(c.n, dtype=torch.float64, device=dev)
        An, bn, _ = c.new_outputs(want_q=False)
        try:
            eec.eec_newton_dc(c.ctx, xd, An, bn, max_iter=1, step_rule=1, solver=solver)
        except eec.EECError:
            pass
        xd.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            its = eec.eec_newton_dc(c.ctx, xd, An, bn, max_iter=300, step_rule=1,
                                    solver=solver)
        except eec.EECError as e:
            out[nname] = {"error": str(e), "s": time.perf_counter() - t0}
            continue
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3
        ev_ms = _time(lambda: c.eval_stamp(xd, An, bn, want_q=False), 20, stream)
        info = eec.eec_newton_info(c.ctx)
        out[nname] = {"unknowns": c.n, "devices": nn.n_dev, "iterations": its,
                      "path": eec.NEWTON_PATHS[info["path"]], "gshunt_stages": info["stages"],
                      "relaxation_sweeps": info["sweeps"],
                      "step_rule": "per-node clip to 0.2 V",
                      "solver": {0: "batched sparse QR, analysis reused",
                                 1: "sparse QR after symmetric AMD ordering",
                                 2: "library sparse LU (static pivots, GPU refactorisation)"}[solver],
                      "lu_stats": eec.eec_lu_stats(c.ctx) if solver == 2 else None, "ms": ms,
                      "ms_per_iteration": ms / max(its, 1), "eval_stamp_ms": ev_ms,
                      "eval_stamp_share": ev_ms * max(its, 1) / ms}
    # the batch of config 4 as one block-diagonal system: the DC points of 4,096 circuits in one
    # Newton loop (its convergence tests take the maximum over every circuit's nodes)
    if time.perf_counter() - t_start < 120:
        nets = netgen.batch_circuits(4096)
        c = eec.Circuit(None, netgen.default_cards(), color=True, batch=nets)
        xd = torch.zeros(c.n, dtype=torch.float64, device=dev)
        An, bn, _ = c.new_outputs(want_q=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            its = eec.eec_newton_dc(c.ctx, xd, An, bn, max_iter=300, step_rule=1, solver=2)
            torch.cuda.synchronize()
            info = eec.eec_newton_info(c.ctx)
            ms = (time.perf_counter() - t0) * 1e3
            out["batch_4096_circuits_solver2"] = {
                "unknowns": c.n, "devices": c.n_dev, "iterations": its,
                "path": eec.NEWTON_PATHS[info["path"]], "relaxation_sweeps": info["sweeps"],
                "lu_stats": eec.eec_lu_stats(c.ctx), "ms": ms, "ms_per_iteration": ms / max(its, 1)}
        except eec.EECError as e:
            out["batch_4096_circuits_solver2"] = {"error": str(e)}
    # NEXT-1 with the GPU Newton loop: transient runs (trapezoidal, fixed step, sources held)
    # from every node at 0 V (power-up: the circuit settles, the chain's stages switch one after
    # another), every step's Newton iterations solved with the library's sparse LU
    for nname, nn, h, steps in (("ripple_adder_64", netgen.ripple_adder(64), 10e-12, 200),
                                ("inverter_chain_1024", netgen.inverter_chain(1024, vin=1.0),
                                 5e-12, 200)):
        key = f"{nname}_transient_tr"
        if time.perf_counter() - t_start > 120:
            out[key] = {"skipped": "time budget of the study used up"}
            continue
        c = eec.Circuit(nn, netgen.default_cards(), color=True)
        xd = torch.zeros(c.n, dtype=torch.float64, device=dev)
        try:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            its = eec.eec_transient(c.ctx, xd, h, steps, method=1, solver=2)
            torch.cuda.synchronize()
        except eec.EECError as e:
            out[key] = {"error": str(e)}
            continue
        ms = (time.perf_counter() - t0) * 1e3
        out[key] = {"unknowns": c.n, "devices": nn.n_dev, "steps": steps, "h_s": h,
                    "newton_iterations": its, "ms": ms, "ms_per_iteration": ms / max(its, 1),
                    "start": "every node at 0 V"}
    return out


def _time(fn, reps, stream):
    import torch
    for _ in range(2):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def extras(eec, circ, net, x, xt, A, b, q, args, dev):
    """The SRAM (high-conflict) step, backward vs plain forward (config 5), per-variant phase
    split (t_calc / t_stamp), the gather's HBM roofline, the transient stamp, the Table II
    adder study, batched vs 4096 separate calls."""
    import torch
    import netgen
    stream = torch.cuda.current_stream()
    res = {}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    # the 256 x 256 6T SRAM: high conflict (512 access transistors per word line, 516 colours)
    sram = netgen.sram(256, 256)
    sc = eec.Circuit(sram, netgen.default_cards(), color=True)
    xs = torch.as_tensor(netgen.random_x(sram), device=dev)
    As, bs, qs = sc.new_outputs()
    ms_s = eec.eec_autotune(sc.ctx, xs, As, bs, qs, reps=5)
    st_ms, _ = timed_steps(eec, sc, xs, As, bs, qs, 200, 10, flush, stream, 1)
    ms = sum(st_ms) / len(st_ms)
    res["sram_256x256"] = {
        "devices": sc.n_dev, "unknowns": sc.n, "colors": sc.n_colors,
        "variant": eec.VARIANT_NAMES[eec.eec_get_variant(sc.ctx)], "ms_per_step": ms,
        "devices_per_s": sc.n_dev / (ms * 1e-3),
        "l2": "flushed (256 MiB write) before every timed step",
        "variants_ms": {eec.VARIANT_NAMES[i]: m for i, m in enumerate(ms_s)}}
    # backward (config 5: the SRAM with gA, gb ~ N(0, 1)) against its plain forward
    rng = netgen.Rng(netgen.DEFAULT_SEED, 12)
    gA = torch.as_tensor(rng.normal(sc.nnz), device=dev)
    gb = torch.as_tensor(rng.normal(sc.n), device=dev)
    gx = torch.empty(sc.n, dtype=torch.float64, device=dev)
    gW = torch.empty(sc.n_dev, dtype=torch.float64, device=dev)
    gL = torch.empty(sc.n_dev, dtype=torch.float64, device=dev)
    fwd_ms = _time(lambda: sc.eval_stamp(xs, As, bs, qs), 50, stream)
    bwd_ms = _time(lambda: eec.eec_eval_stamp_bwd(sc.ctx, xs, gA, gb, gx, gW, gL), 20, stream)
    res["bwd"] = {"devices_per_s": sc.n_dev / (bwd_ms * 1e-3), "ms": bwd_ms,
                  "fwd_ms": fwd_ms, "bwd_over_fwd_time": bwd_ms / fwd_ms,
                  "workload": "config 5: SRAM 256x256, gA, gb ~ N(0, 1)"}
    del sc
    phases = {}
    v0 = eec.eec_get_variant(circ.ctx)
    for v in range(eec.EEC_N_VARIANTS):
        eec.eec_set_variant(circ.ctx, v)
        eec.eec_profile_enable(circ.ctx, True)
        eec.eec_profile_read(circ.ctx)
        for _ in range(10):
            circ.eval_stamp(xt, A, b, q)
        p = eec.eec_profile_read(circ.ctx)
        eec.eec_profile_enable(circ.ctx, False)
        n = max(p["calls"], 1)
        phases[eec.VARIANT_NAMES[v]] = {"init_ms": p["ms_init"] / n, "eval_ms": p["ms_eval"] / n,
                                        "stamp_ms": p["ms_stamp"] / n}
    eec.eec_set_variant(circ.ctx, v0)
    res["phases_ungraphed"] = phases

    # HBM roofline of the stamp-only kernel (the segmented-reduction gather from the buffer in
    # entry order): per contribution its 8 B value, per A/b entry 8 B of its linear part and 8 B
    # written (the chunk descriptors, 16 B per 64 items, and the unused ends of chunks not
    # counted)
    _, _, unk = circ.pattern()
    free = unk[net.dev_nodes] >= 0
    contrib = int((free[:, [0, 2, 3]].sum(axis=1) * (1 + free.sum(axis=1))).sum())
    entries = circ.nnz + circ.n
    gbytes = 8 * contrib + 16 * entries
    st_ms = phases["segreduce"]["stamp_ms"]
    hbm = hbm_peak_gbs()
    res["stamp_roofline"] = {
        "kernel": "k_gather (segmented-reduction stamp)", "bound": "hbm",
        "achieved": gbytes / (st_ms * 1e-3) / 1e9, "peak": hbm[0], "unit": "GB/s",
        "frac": gbytes / (st_ms * 1e-3) / 1e9 / hbm[0], "algorithmic_bytes": gbytes,
        "contributions": contrib, "entries": entries, "peak_source": hbm[1],
        "workload": "the bench's workload",
        "note": "the buffer is read right after the evaluate kernel wrote it (15 doubles per "
                "device: partly L2-resident)"}

    # transient companion stamp (trapezoidal rule) on the same workload
    qprev = torch.empty_like(q)
    circ.eval_stamp(xt, A, b, qprev)
    ic = torch.empty_like(q)
    ip = torch.zeros_like(q)
    v0t = eec.eec_get_variant(circ.ctx)
    tran = {}
    for v in (eec.EEC_VARIANT_ATOMIC, eec.EEC_VARIANT_COLOR_FUSED, eec.EEC_VARIANT_COLOR_BUFFERED,
              eec.EEC_VARIANT_COLOR_PIPELINED):
        eec.eec_set_variant(circ.ctx, v)
        ms_t = _time(lambda: eec.eec_eval_stamp_tran(circ.ctx, xt, qprev, ip, 2e11, 1.0, A, b, q, ic),
                     3 if v == eec.EEC_VARIANT_COLOR_FUSED else 20, stream)
        tran[eec.VARIANT_NAMES[v]] = {"ms": ms_t, "devices_per_s": net.n_dev / (ms_t * 1e-3)}
    eec.eec_set_variant(circ.ctx, v0t)
    res["transient_tr_stamp"] = tran


    # Table II analogue: 64-bit ripple-carry adder (28T mirror full adders), with 14 series
    # resistors per bit and with every transistor-to-transistor connection split, coloured by the
    # free-node rule (0) and the literal any-non-ground rule (1, VDD counted)
    cards0 = netgen.default_cards()
    base = netgen.ripple_adder(64)
    study = {}
    for name, n in (("base", base), ("R14", netgen.insert_series_resistors(base, per_group=14)),
                    ("R_all", netgen.insert_series_resistors(base))):
        for rule in (0, 1):
            c = eec.Circuit(n, cards0, color=True, conflict_rule=rule)
            xa = torch.as_tensor(netgen.random_x(n), device=dev)
            A2, b2, q2 = c.new_outputs()
            msv = eec.eec_autotune(c.ctx, xa, A2, b2, q2, reps=5)
            study[f"{name}_rule{rule}"] = {
                "transistors": n.n_dev, "resistors": int(len(n.res_G)), "colors": c.n_colors,
                "ms": {eec.VARIANT_NAMES[i]: m for i, m in enumerate(msv)}}
            del c
    # the same netlists in modified nodal analysis (rails and their source currents are
    # unknowns): the free-node rule then sees the VDD clique, the reading that gives Table II's
    # 896 colours with real stamping
    for name, n in (("base", base), ("R14", netgen.insert_series_resistors(base, per_group=14))):
        c = eec.Circuit(n, cards0, color=True, rail_mode=eec.EEC_RAIL_MNA_BRANCH)
        xm = np.concatenate([netgen.Rng(7, 8).uniform(n.n_nodes - 1),
                             1e-4 * netgen.Rng(7, 9).normal(c.n - n.n_nodes + 1)])
        xa = torch.as_tensor(xm, device=dev)
        A2, b2, q2 = c.new_outputs()
        msv = eec.eec_autotune(c.ctx, xa, A2, b2, q2, reps=5)
        study[f"{name}_mna_rule0"] = {
            "transistors": n.n_dev, "resistors": int(len(n.res_G)), "colors": c.n_colors,
            "unknowns": c.n, "ms": {eec.VARIANT_NAMES[i]: m for i, m in enumerate(msv)}}
        del c
    res["adder64_table2_study"] = study

    # batched (config 4): one context for 4096 circuits vs 4096 plain per-circuit calls
    nets = netgen.batch_circuits(4096)
    cards = netgen.default_cards()
    bc = eec.Circuit(None, cards, color=True, batch=nets)
    xb = torch.as_tensor(netgen.random_x(netgen.concat(nets)), device=dev)
    Ab, bb_, qb = bc.new_outputs()
    ms_b = eec.eec_autotune(bc.ctx, xb, Ab, bb_, qb, reps=5)
    vb = eec.eec_get_variant(bc.ctx)
    eec.eec_graph_capture(bc.ctx, xb, Ab, bb_, qb)
    t_graph = _time(lambda: eec.eec_graph_launch(bc.ctx), 20, stream)
    t_batch = _time(lambda: bc.eval_stamp(xb, Ab, bb_, qb), 20, stream)
    ro, no, do = eec.eec_get_batch_offsets(bc.ctx, len(nets))
    plain = [eec.Circuit(m, cards, color=True, variant=vb) for m in nets]
    views = []
    for k, c in enumerate(plain):
        views.append((xb[ro[k]:ro[k + 1]], Ab[no[k]:no[k + 1]], bb_[ro[k]:ro[k + 1]],
                      torch.empty(4 * c.n_dev, dtype=torch.float64, device=dev)))

    def all_plain():
        for c, (xv, av, bv, qv) in zip(plain, views):
            c.eval_stamp(xv, av, bv, qv)
    t_plain = _time(all_plain, 3, stream)
    nd = bc.n_dev
    res["batched"] = {"circuits": len(nets), "devices": nd, "colors_merged": bc.n_colors,
                      "variant": eec.VARIANT_NAMES[vb],
                      "batched_devices_per_s": nd / (t_batch * 1e-3),
                      "graph_devices_per_s": nd / (t_graph * 1e-3),
                      "plain_4096_calls_devices_per_s": nd / (t_plain * 1e-3),
                      "batched_ms": t_batch, "graph_ms": t_graph, "plain_4096_calls_ms": t_plain,
                      "speedup_vs_plain": t_plain / t_graph,
                      "variants_ms": {eec.VARIANT_NAMES[i]: m for i, m in enumerate(ms_b)}}
    del plain
    return res


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.newton:
        import torch
        import paper_2604_03079_gb300 as eec
        dev = torch.device("cuda", torch.cuda.current_device())
        print(json.dumps({"newton_dc_gpu": newton_study(eec, dev, torch.cuda.current_stream())}))
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
