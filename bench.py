"""Throughput of the loop-hafnian sieve on GB300 (one JSON line on rank 0).

Headline workload (default, ``--workload large60``): ONE whole 60-photon collision-free loop
hafnian (100-mode Haar kernel, r ~ U[1.2,1.8], complex-normal loops, complex128), 2^29 evaluated
sieve terms of working dimension 61. The K timed steps are K contiguous term ranges that together
cover every term exactly once (``lhaf_range`` with device inputs; inside a step the library runs
bounded launches of about a quarter second each); their double-double partials are combined at the
end into the loop hafnian. ms per 60-photon lhaf = the sum of the K step times; value = terms / that
time. Warm-up steps run on separate small slices of the same sum and are not counted. The L2 is
flushed (256 MiB write) between steps, outside the step events.

``--workload collision40``: every step is one whole 40-photon collision-pattern loop hafnian (100
modes, 40 photons over 22 modes with counts 1..4, gamma = 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload large60|collision40] [--terms T] [--no-extras] [--no-cpu-baseline]

``--terms T`` restricts the timed steps to the first T terms (profiling runs; the line then says
so). N > 1 runs under torchrun, one rank per GPU: the term ranges of the one loop hafnian are split
over the ranks (``sharded.term_shard``), each rank's partial moves in one all-gather, and every rank
combines the same value (strong scaling).
"""
from __future__ import annotations

import argparse
import hashlib
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

UNIT = "terms/s"
WORKLOADS = {
    "large60": dict(
        metric="lhaf sieve terms/s of one whole 60-photon loop hafnian (FP64); ms per 60-photon lhaf",
        desc=("60-photon collision-free loop hafnian: 100-mode Haar interferometer, r ~ U[1.2,1.8], complex-normal "
              "loop weights (E|gamma|^2 = 0.5), 60 distinct modes with one photon each, complex128, finite difference "
              "sieve with double-double accumulation")),
    "collision40": dict(
        metric="lhaf sieve terms/s (collision-pattern loop hafnian, FP64)",
        desc=("collision-pattern loop hafnian: 100-mode Haar interferometer, r ~ U[1.0,1.6], gamma = 0, 40 photons "
              "over 22 modes with counts 1..4 (seeded multinomial), complex128, repeated-pair sieve")),
}
# FP64 peak: no FP64 figure is measured by the pool, so it is derived from unit counts and the clock
NOMINAL_FP64_TFLOPS = 152 * 4 * 0.5 * 2 * 2.070 / 1e3  # SMs x sub-partitions x FMA lanes/clk x 2 x GHz
PEAK_SOURCE = "derived: 152 SMs x 4 sub-partitions x 0.5 FP64 FMA lanes/clk x 2 flops x 2.070 GHz"
# DRAM traffic (read + write bytes) per launch of the dominant kernel, from one ncu capture of a
# full-size launch, valid only for the kernel source it was taken on (else reported as null)
KERNEL_TRAFFIC = {
    # workload: (sha256[:16] of csrc/lhaf_terms.cu at capture, bytes of the captured launch, its terms)
    "large60": ("ac3da7541ec2bfa6", 437760 + 57118208, 110557),
    "collision40": ("ac3da7541ec2bfa6", 223488 + 0, 34560),
}


def rank_info():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def kernel_source_sha() -> str:
    with open(os.path.join(ROOT, "paper_2108_01622_gb300", "csrc", "lhaf_terms.cu"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def load_problem(workload: str):
    from paper_2108_01622_gb300 import workloads as wl

    return wl.large_lhaf_60(seed=5) if workload == "large60" else wl.collision_lhaf_40(seed=2)


def survey_flops_per_term(n: int, h: int) -> float:
    """The fixed model F(n, h) = (40/3) n^3 + (4/3) n^3 + 8 min(h-1, n) n^2 + 8 h^2 (Householder
    reduction, La Budde, loop products, series), n the slot count (the border not counted)."""
    return (40.0 / 3.0 + 4.0 / 3.0) * n ** 3 + 8.0 * min(h - 1, n) * n ** 2 + 8.0 * h ** 2


# ------------------------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm): the oracle as it stands, on a bounded
# sample of the same workload's sieve terms, over the host cores. The oracle sums every digit
# vector; its first half (first digit below the middle) is the half the library evaluates, term
# for term of the same cost, so its terms/s is in the same units and ms per lhaf = (evaluated
# terms) / rate.
# ------------------------------------------------------------------------------------------


class OracleTimer:
    """The C oracle as it stands (Householder Hessenberg form, La Budde's recurrence, Newton's
    identities; OpenMP over terms on every host core), timed on slices of the workload's sieve
    terms."""

    def __init__(self, workload: str):
        from oracle import csieve
        from oracle import lhaf_oracle as lo

        self.cs = csieve
        self.p = load_problem(workload)
        self.total_terms = lo.repeated_term_count(self.p.reps)
        self.half = max(1, self.total_terms // 2)
        _, self.cores = csieve.sieve_sum(self.p.B, self.p.gamma, self.p.reps, 0, 64)  # builds, warms up
        n = min(self.half, 16 * self.cores)
        t0 = time.perf_counter()
        csieve.sieve_sum(self.p.B, self.p.gamma, self.p.reps, 0, n)
        self.per_term = (time.perf_counter() - t0) / n
        self.cursor = n

    def sample(self, seconds: float, evaluated_terms: int):
        n = max(4 * self.cores, int(seconds / self.per_term))
        n = min(n, self.half)
        if self.cursor + n > self.half:
            self.cursor = 0
        t0 = time.perf_counter()
        _, used = self.cs.sieve_sum(self.p.B, self.p.gamma, self.p.reps, self.cursor, self.cursor + n)
        wall = time.perf_counter() - t0
        self.cursor += n
        self.per_term = wall / n
        rate = n / wall
        return {"value": rate, "unit": UNIT, "cores": used, "kind": "oracle",
                "sample": (f"{n} sieve terms of the same workload (a contiguous slice of the half the library "
                           f"evaluates; {self.total_terms} digit vectors in all), C oracle (Householder Hessenberg, "
                           f"La Budde, Newton; FP64, long-double sums), OpenMP over terms on {used} threads, "
                           f"{wall:.1f} s wall"),
                "ms_per_lhaf": evaluated_terms / rate * 1e3}

    def close(self):
        pass


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------

CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, index: int):
        self.dir = tempfile.mkdtemp(prefix="lhaf_clocks_")
        self.path = os.path.join(self.dir, f"clocks_gpu{index}.csv")
        self.proc = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={CLOCK_FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def evaluated_terms(workload: str) -> int:
    import paper_2108_01622_gb300 as lg

    p = load_problem(workload)
    loops = bool(np.any(np.asarray(p.gamma)[np.asarray(p.reps) > 0] != 0))
    return lg.plan(p.reps, has_loops=loops)[0]


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    meta = WORKLOADS[args.workload]
    timer = OracleTimer(args.workload)
    T = timer.half  # the halved sum: the terms the library evaluates for these workloads
    per_step = min(10.0, max(0.3, 150.0 / (args.steps + args.warmup)))
    rates = []
    base = None
    for s in range(args.warmup + args.steps):
        r = timer.sample(per_step, T)
        if s >= args.warmup:
            rates.append(r["value"])
        base = r
    timer.close()
    value = statistics.median(rates)
    line = {"impl": "reference", "metric": meta["metric"], "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": T / args.steps / value * 1e3,
            "ms_per_lhaf": T / value * 1e3, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": meta["desc"], "evaluated_terms": T, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": base["cores"], "kind": "oracle",
                             "sample": base["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def rank_step_ranges(T: int, rank: int, world: int, steps: int):
    """The `steps` contiguous term ranges of `rank`: its share of [0, T) (``sharded.term_shard``)
    cut into near-equal pieces; over all ranks and steps they cover [0, T) once, in term order."""
    from paper_2108_01622_gb300 import sharded

    rb, re_ = sharded.term_shard(T, rank, world)
    cuts = [rb + (re_ - rb) * s // steps for s in range(steps + 1)]
    return [(cuts[s], cuts[s + 1]) for s in range(steps)]


def _ev(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def run_ours(args, rank, world, local_rank):
    import torch

    import paper_2108_01622_gb300 as lg
    from paper_2108_01622_gb300 import sharded

    meta = WORKLOADS[args.workload]
    p = load_problem(args.workload)
    loops = bool(np.any(np.asarray(p.gamma)[np.asarray(p.reps) > 0] != 0))
    T_all, nd, h, P = lg.plan(p.reps, has_loops=loops)
    groups = lg.plan_groups(p.reps, has_loops=loops)
    whole_sum = args.workload == "large60"
    T_timed = T_all if (args.terms is None or not whole_sum) else max(1, min(int(args.terms), T_all))

    cpu_base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        timer = OracleTimer(args.workload)  # before the first GPU call
        cpu_base = timer.sample(15.0, T_all)
        timer.close()

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    ctx = lg.Context(local_rank)  # ordered on torch's current stream
    Bd = torch.from_numpy(p.B).to(dev)
    gd = torch.from_numpy(p.gamma).to(dev)
    flags = 0 if loops else lg.NO_LOOPS
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    fp64_gflops = lg.fp64_probe(local_rank)

    # this rank's share of the timed terms, cut into `steps` contiguous ranges
    if whole_sum:
        ranges = rank_step_ranges(T_timed, rank, world, args.steps)
        wsz = min(1 << 13, T_all)
        warm = [(max(0, T_all - wsz * (w + 1)), max(0, T_all - wsz * (w + 1)) + wsz) for w in range(args.warmup)]
    out = torch.empty(1, dtype=torch.complex128, device=dev)
    for w in range(args.warmup):
        if whole_sum:
            ctx.lhaf_range(Bd, gd, p.reps, warm[w][0], warm[w][1], flags=flags)
        else:
            ctx.lhaf(Bd, gd, p.reps, flags=flags, out=out)
    torch.cuda.synchronize()

    evs = [_ev(torch) for _ in range(args.steps)]
    kern_ms, flops, term_launches, launches, parts = [], 0.0, 0, 0, []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank)
    time.sleep(0.3)
    for s in range(args.steps):
        flush.zero_()
        evs[s][0].record()
        if whole_sum:
            part, st = ctx.lhaf_range(Bd, gd, p.reps, ranges[s][0], ranges[s][1], flags=flags, stats=True)
            parts.append(part)
        else:
            _, st = ctx.lhaf(Bd, gd, p.reps, flags=flags, out=out, stats=True)
        evs[s][1].record()
        kern_ms.append(st["kernel_ms"])
        flops += st["flops_model"]
        term_launches += st["term_launches"]
        launches += st["launches"]
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    if whole_sum:
        mine = torch.stack(parts).cpu().numpy()
        allp = sharded.gather_partials(mine) if world > 1 else mine
        val = lg.combine(allp, h) if T_timed == T_all else None
        value = T_timed / (total_ms * 1e-3)
        ms_lhaf = total_ms * T_all / T_timed
    else:
        val = complex(out.cpu()[0])
        value = world * args.steps * T_all / (total_ms * 1e-3)
        ms_lhaf = total_ms / args.steps

    # e2e: the public host-pointer call (pinned staging copies inside the library), timed on the host
    e2e_terms, e2e_s, h2d, d2h, e2e_calls = 0, 0.0, 0, 0, 0
    if whole_sum:
        n_e = min(T_timed, 1 << 20)
        ctx.lhaf_range(p.B, p.gamma, p.reps, 0, min(n_e, 1 << 12))
        for c in range(3):
            b0 = (c * n_e) % max(1, T_all - n_e + 1)
            t0 = time.perf_counter()
            _, est = ctx.lhaf_range(p.B, p.gamma, p.reps, b0, b0 + n_e, stats=True)
            e2e_s += time.perf_counter() - t0
            e2e_terms += n_e
            h2d, d2h, e2e_calls = est["h2d_bytes"], est["d2h_bytes"], e2e_calls + 1
        e2e = {"value": e2e_terms / e2e_s, "unit": UNIT, "ms_per_lhaf_projected": T_all / (e2e_terms / e2e_s) * 1e3,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "sample": f"{e2e_calls} host-pointer lhaf_range calls of {n_e} terms each (inputs copied from host "
                         f"memory and the 4-double partial copied back inside every call)"}
    else:
        _, est = ctx.lhaf(p.B, p.gamma, p.reps, stats=True)
        ts = []
        for _ in range(max(3, args.steps // 4)):
            t0 = time.perf_counter()
            ctx.lhaf(p.B, p.gamma, p.reps)
            ts.append(time.perf_counter() - t0)
        e2e_ms = statistics.median(ts) * 1e3
        e2e = {"value": T_all / (e2e_ms * 1e-3), "unit": UNIT, "ms_per_lhaf": e2e_ms,
               "h2d_bytes_per_step": est["h2d_bytes"], "d2h_bytes_per_step": est["d2h_bytes"]}

    extras = {} if (args.no_extras or world > 1) else run_extras(ctx, torch, dev, lg, args.workload)

    # roofline of the dominant kernel (the sieve terms): model flops over its launches' device time
    kern_total = sum(kern_ms)
    achieved = flops / (kern_total * 1e-3) / 1e12
    n_slots = nd - (1 if loops else 0)
    survey_flops = survey_flops_per_term(n_slots, h) * (T_timed if whole_sum else T_all * args.steps)
    tr = KERNEL_TRAFFIC.get(args.workload)
    traffic = None
    if tr and tr[0] == kernel_source_sha():
        # the captured launch's DRAM bytes scaled to this run's average launch by its terms (the
        # traffic is the staged term polynomials, proportional to the terms of a launch)
        terms_per_launch = (T_timed if whole_sum else T_all * args.steps) / max(term_launches, 1)
        traffic = tr[1] * terms_per_launch / tr[2]
    roofline = {"bound": "alu", "kernel": "grouped_terms_kernel (FP64 sieve terms)", "achieved": achieved,
                "peak": NOMINAL_FP64_TFLOPS, "unit": "TFLOP/s", "frac": achieved / NOMINAL_FP64_TFLOPS,
                "traffic": traffic, "peak_source": PEAK_SOURCE + " (no FP64 entry is measured by the pool)",
                "fp64_probe_tflops": fp64_gflops / 1e3, "frac_of_probe": achieved / (fp64_gflops / 1e3),
                "flops_per_launch": flops / max(term_launches, 1), "avg_launch_ms": kern_total / max(term_launches, 1),
                "launches": term_launches,
                "flop_model": ("implementation: 8 flops per complex multiply-add of the elimination reduction, La "
                               "Budde tables and series actually executed (lhaf_flops_per_term)"),
                "survey_model_frac": survey_flops / (kern_total * 1e-3) / 1e12 / NOMINAL_FP64_TFLOPS,
                "survey_model_note": ("F(n,h) = (40/3+4/3) n^3 + 8 min(h-1,n) n^2 + 8 h^2 assumes a Householder "
                                      "reduction (twice the elimination's flops) and separate loop products; "
                                      "above 1 for this kernel, so the implementation model is the reported frac"),
                "traffic_note": ("DRAM read + write bytes of one launch from an ncu capture of the current kernel "
                                 "source, scaled to the average launch by its terms" if traffic is not None
                                 else "no ncu capture of the current kernel source")}
    cfg = {"workload": meta["desc"], "evaluated_terms": T_all, "timed_terms": T_timed, "n_dim": nd, "h": h,
           "pairs": P, "team": st["team"], "zero_digit_groups": groups,
           "l2": "flushed between steps (256 MiB write, outside step events)",
           "parallelism": (f"term ranges of one loop hafnian over {world} GPU(s)" if whole_sum else
                           f"{world} independent loop hafnians, one per GPU")}
    if whole_sum:
        cfg["steps_cover"] = ("all terms of one loop hafnian, each exactly once, in contiguous ranges" if T_timed == T_all
                              else f"the first {T_timed} of {T_all} terms (partial run)")
    line = {
        "metric": meta["metric"], "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "strong" if whole_sum else "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": cfg, "gpu_launches": launches, "roofline": roofline, "e2e": e2e, "clocks": clocks,
    }
    if whole_sum and T_timed == T_all:
        line["ms_per_60_photon_lhaf"] = ms_lhaf
    elif whole_sum:
        line["ms_per_60_photon_lhaf_projected"] = ms_lhaf
    else:
        line["ms_per_lhaf"] = ms_lhaf
    if val is not None:
        line["result"] = [val.real, val.imag]
    line.update(extras)
    if cpu_base is not None:
        line["cpu_baseline"] = {k: cpu_base[k] for k in ("value", "unit", "cores", "kind", "sample")}
        line["cpu_baseline"]["ms_per_lhaf"] = cpu_base["ms_per_lhaf"]
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def _timed(torch, fn, reps=3):
    """Median device time (ms) of fn() over reps calls (CUDA events on the current stream)."""
    times = []
    for _ in range(reps):
        a, b = _ev(torch)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    return statistics.median(times)


def run_extras(ctx, torch, dev, lg, workload):
    """The rest of the metric, each on its own workload (untimed by the step loop above): the
    40-photon collision pattern one call at a time, the 60-photon slice with plain FP64
    accumulation, batched vs one call per item on the 4096-item chain-rule batch, the batched
    mode of one chain-rule step, loop-vector sharing, a chain-rule step, a mixed-state
    probability, the eigenvalue-trace accuracy comparison and the adjoint."""
    from paper_2108_01622_gb300 import workloads as wl

    out = {}

    def _collision40_and_plain_accum():
        if workload == "large60":
            # the 40-photon collision pattern (100 modes, counts 1..4, gamma = 0): whole calls
            p = wl.collision_lhaf_40(seed=2)
            T, nd, h, _ = lg.plan(p.reps, has_loops=False)
            Bd = torch.from_numpy(p.B).to(dev)
            gd = torch.from_numpy(p.gamma).to(dev)
            o = torch.empty(1, dtype=torch.complex128, device=dev)
            ctx.lhaf(Bd, gd, p.reps, flags=lg.NO_LOOPS, out=o)
            ks, fl = [], 0.0
            for _ in range(10):
                _, st = ctx.lhaf(Bd, gd, p.reps, flags=lg.NO_LOOPS, out=o, stats=True)
                ks.append(st["kernel_ms"])
                fl = st["flops_model"]
            ms = _timed(torch, lambda: ctx.lhaf(Bd, gd, p.reps, flags=lg.NO_LOOPS, out=o), reps=10)
            out["collision40"] = {"workload": WORKLOADS["collision40"]["desc"], "terms": T, "n_dim": nd, "h": h,
                                  "ms_per_lhaf": ms, "terms_per_s": T / (ms * 1e-3),
                                  "kernel_tflops": fl / (statistics.median(ks) * 1e-3) / 1e12,
                                  "kernel_frac": fl / (statistics.median(ks) * 1e-3) / 1e12 / NOMINAL_FP64_TFLOPS}
            # plain FP64 accumulation against double-double on a 2^17-term slice of the 60-photon sum
            p60 = wl.large_lhaf_60(seed=5)
            S = 1 << 17
            pd = ctx.lhaf_range(p60.B, p60.gamma, p60.reps, 0, S)
            pp = ctx.lhaf_range(p60.B, p60.gamma, p60.reps, 0, S, flags=lg.PLAIN_ACCUM)
            sd, sp = complex(pd[0] + pd[1], pd[2] + pd[3]), complex(pp[0] + pp[1], pp[2] + pp[3])
            out["lhaf60_plain_accum"] = {"slice_terms": S, "plain_vs_dd_rel_diff": abs(sp - sd) / abs(sd)}

    def _batched():
        # batched vs one call per item: the 4096 loop hafnians of the chain-rule batch (N in 10..40)
        b = wl.chain_rule_batch(seed=3, count=4096)
        R = np.array(b.reps)
        Gd = torch.from_numpy(np.array(b.gammas)).to(dev)
        Bd = torch.from_numpy(b.B).to(dev)
        ob = torch.empty(len(R), dtype=torch.complex128, device=dev)
        op = torch.empty(len(R), dtype=torch.complex128, device=dev)
        og = torch.empty(len(R), dtype=torch.complex128, device=dev)
        ctx.lhaf_batched(Bd, Gd, R, out=ob)

        def plain():
            for i in range(len(R)):
                ctx.lhaf(Bd, Gd[i], R[i], out=op[i:i + 1])

        plain()  # warms the per-shape tuning cache of the single-call path
        torch.cuda.synchronize()
        tb = _timed(torch, lambda: ctx.lhaf_batched(Bd, Gd, R, out=ob), reps=1)
        tp = _timed(torch, plain, reps=1)
        with ctx.batched_plan(Bd, Gd, R) as plan:
            plan.run(Bd, Gd, out=og)
            tg_ = _timed(torch, lambda: plan.run(Bd, Gd, out=og), reps=1)
        d = torch.maximum((ob - op).abs() / op.abs(), (og - op).abs() / op.abs())
        # the most cancelling items against the C oracle's long double values (tests/golden): an FP64
        # sum keeps about 16 - log10(condition) digits, whichever form evaluates it
        ill = []
        gpath = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden",
                             "chain_rule_ill_conditioned.json")
        if os.path.exists(gpath):
            with open(gpath) as f:
                for it in json.load(f)["items"]:
                    i, ref = it["index"], complex(*it["value"])
                    e = {k: abs(complex(v[i].item()) - ref) / abs(ref) for k, v in (("batched", ob), ("plain", op),
                                                                                    ("graph", og))}
                    ill.append({"index": i, "photons": it["photons"], "condition": it["condition"],
                                "bound_cond_x_2^-52": it["condition"] * 2.0 ** -52,
                                "rel_err_batched": e["batched"], "rel_err_plain": e["plain"],
                                "rel_err_graph": e["graph"],
                                "rel_err_fp64_c_oracle": abs(complex(*it["fp64_c_oracle"]) - ref) / abs(ref)})
        out["batched"] = {"workload": "chain-rule batch: 4096 loop hafnians, 50-mode lossy GBS state, N~U{10..40}",
                          "batched_ms": tb, "graph_replay_ms": tg_, "plain_ms": tp,
                          "batched_over_plain_speedup": tp / tb, "graph_over_plain_speedup": tp / tg_,
                          "max_rel_diff": float(d.max().item()),
                          "items_rel_diff_over_1e-10": int((d > 1e-10).sum().item()),
                          "ill_conditioned_items_vs_extended_oracle": ill}

    def _batched_small():
        # small items only: many short loop hafnians, where one launch per item is launch-bound
        bs = wl.chain_rule_batch(seed=7, count=2048, n_lo=8, n_hi=16)
        Rs = np.array(bs.reps)
        Gs = torch.from_numpy(np.array(bs.gammas)).to(dev)
        Bs = torch.from_numpy(bs.B).to(dev)
        obs = torch.empty(len(Rs), dtype=torch.complex128, device=dev)
        ops_ = torch.empty(len(Rs), dtype=torch.complex128, device=dev)
        ctx.lhaf_batched(Bs, Gs, Rs, out=obs)

        def plain_s():
            for i in range(len(Rs)):
                ctx.lhaf(Bs, Gs[i], Rs[i], out=ops_[i:i + 1])

        plain_s()
        tbs = _timed(torch, lambda: ctx.lhaf_batched(Bs, Gs, Rs, out=obs), reps=2)
        tps = _timed(torch, plain_s, reps=2)
        ogs = torch.empty(len(Rs), dtype=torch.complex128, device=dev)
        with ctx.batched_plan(Bs, Gs, Rs) as plan:
            plan.run(Bs, Gs, out=ogs)
            tgs = _timed(torch, lambda: plan.run(Bs, Gs, out=ogs), reps=3)
        out["batched_small"] = {"workload": "2048 loop hafnians, N~U{8..16}, same state family",
                                "batched_ms": tbs, "graph_replay_ms": tgs, "plain_ms": tps,
                                "batched_over_plain_speedup": tps / tbs, "graph_over_plain_speedup": tps / tgs}

    def _batched_mode():
        # batched mode of one chain-rule step (App. B.5): the next mode's outcomes n = 0..8 at once,
        # against the same nine loop hafnians as one batch
        cb = wl.chain_rule_batch(seed=11, count=64, n_lo=26, n_hi=30)
        ci = max(range(len(cb.reps)), key=lambda i: int(np.sum(cb.reps[i])))
        fixed = np.array(cb.reps[ci], dtype=np.int32)
        mode = int(np.nonzero(fixed == 0)[0][0])
        gm = np.array(cb.gammas[ci])
        n_cut = 8
        pats = np.repeat(fixed[None, :], n_cut + 1, axis=0)
        pats[:, mode] = np.arange(n_cut + 1)
        gms = np.repeat(gm[None, :], n_cut + 1, axis=0)
        ctx.lhaf_batched_mode(cb.B, gm, fixed, mode, n_cut)
        ctx.lhaf_batched(cb.B, gms, pats)
        tm = _timed(torch, lambda: ctx.lhaf_batched_mode(cb.B, gm, fixed, mode, n_cut), reps=3)
        tbp = _timed(torch, lambda: ctx.lhaf_batched(cb.B, gms, pats), reps=3)
        # the costliest single outcome (not necessarily the last: an odd count can add a pair)
        t_each = []
        for pat in pats:
            ctx.lhaf(cb.B, gm, pat)
            t_each.append(_timed(torch, lambda: ctx.lhaf(cb.B, gm, pat), reps=3))
        tl = max(t_each)
        vm = ctx.lhaf_batched_mode(cb.B, gm, fixed, mode, n_cut)
        vb, _ = ctx.lhaf_batched(cb.B, gms, pats)
        out["batched_mode"] = {"workload": f"chain-rule step: {int(fixed.sum())} fixed photons, outcomes 0..{n_cut} "
                                           "of the next mode, 50-mode lossy state",
                               "batched_mode_ms": tm, "batched_patterns_ms": tbp, "speedup": tbp / tm,
                               "largest_outcome_alone_ms": tl, "batched_mode_over_largest": tm / tl,
                               "each_outcome_alone_ms": t_each, "sum_of_outcomes_alone_ms": sum(t_each),
                               "max_rel_diff": float(np.max(np.abs(vm - vb) / np.abs(vb)))}

    def _multi_gamma():
        # several loop-weight vectors on one pattern (App. B.5, threshold sub-detectors): 4, 16 and 64
        # vectors on the 40-photon collision pattern, each against the same loop hafnians as one batch
        pm_ = wl.collision_lhaf_40(seed=2)
        res = {"workload": "4, 16 and 64 loop-weight vectors on the 40-photon collision pattern (100-mode Haar)"}
        for ng in (4, 16, 64):
            Gm = wl.complex_normal(np.random.default_rng(21), (ng, len(pm_.reps)))
            Rm = np.repeat(np.asarray(pm_.reps)[None, :], ng, axis=0)
            vm_ = ctx.lhaf_multi_gamma(pm_.B, Gm, pm_.reps)
            vb_, _ = ctx.lhaf_batched(pm_.B, Gm, Rm)
            tmg = _timed(torch, lambda: ctx.lhaf_multi_gamma(pm_.B, Gm, pm_.reps), reps=3)
            tbg = _timed(torch, lambda: ctx.lhaf_batched(pm_.B, Gm, Rm), reps=3)
            res[str(ng)] = {"multi_gamma_ms": tmg, "batched_ms": tbg, "speedup": tbg / tmg,
                            "max_rel_diff": float(np.max(np.abs(vm_ - vb_) / np.abs(vb_)))}
        out["multi_gamma"] = res

    def _chain_rule_step():
        # one chain-rule step (App. A.2): a 50-mode pure state, 20 photons sampled on half of the
        # modes, coherent amplitudes on the rest, the next mode's distribution over 0..8
        rng_c = np.random.default_rng(31)
        Uc = wl.haar_unitary(rng_c, 50)
        rc = rng_c.uniform(0.8, 1.2, size=50)
        ac = wl.complex_normal(rng_c, 50, 0.1)
        nc = np.zeros(50, dtype=np.int32)
        nc[:25] = wl.pattern_multinomial(rng_c, 25, 20, 3)
        bc = wl.complex_normal(rng_c, 50, 1.0)
        bc[:26] = 0.0
        ctx.gbs_chain_rule_step(Uc, rc, ac, bc, nc, 25, 8, u=0.5)
        tcs = _timed(torch, lambda: ctx.gbs_chain_rule_step(Uc, rc, ac, bc, nc, 25, 8, u=0.5), reps=3)
        out["chain_rule_step"] = {"workload": "50-mode pure state, 20 photons on modes 0..24, coherent amplitudes on "
                                              "26..49, distribution of mode 25 over 0..8 and one draw",
                                  "ms": tcs}

    def _mixed():
        # mixed state (App. B.2 lhafmix): a 20-photon outcome of a 50-mode lossy state, the loop
        # hafnian of the 100 x 100 matrix A with every occupied index pair repeated
        ms_ = wl.lossy_state(seed=12, M=50, r_lo=0.8, r_hi=1.4, eta=0.6)
        nm = wl.pattern_multinomial(np.random.default_rng(12), 50, 20, 3)
        Tm, ndm, hm, _ = lg.plan(np.concatenate([nm, nm]))
        ctx.gbs_pattern_prob_mixed(ms_.sigma, ms_.alpha, nm)
        tmx = _timed(torch, lambda: ctx.gbs_pattern_prob_mixed(ms_.sigma, ms_.alpha, nm), reps=3)
        out["mixed"] = {"workload": "P(n) of a 20-photon outcome (counts <= 3) of a 50-mode lossy state, eta = 0.6",
                        "terms": Tm, "n_dim": ndm, "h": hm, "ms": tmx}

    def _et_vs_fds():
        # eigenvalue-trace variant against the finite difference sieve (App. B.4, Fig. glynn_accuracy):
        # relative error of lhaf(A1 (+) A2) against lhaf(A1) lhaf(A2) (halves by the sieve, each pair
        # crossing the blocks), and the time of one N = 40 loop hafnian by each
        acc = {}
        for n_half in (12, 16, 20):
            ef, ee, epl = [], [], []
            for sd in range(5):
                bp = wl.block_diagonal_pair(seed=1000 * n_half + sd, n=n_half)
                ones_h = [1] * n_half
                ref = ctx.lhaf(bp.A1, None, ones_h) * ctx.lhaf(bp.A2, None, ones_h)
                ones = [1] * (2 * n_half)
                ef.append(abs(ctx.lhaf(bp.C, None, ones) - ref) / abs(ref))
                ee.append(abs(ctx.lhaf(bp.C, None, ones, flags=lg.ET) - ref) / abs(ref))
                epl.append(abs(ctx.lhaf(bp.C, None, ones, flags=lg.PLAIN_ACCUM) - ref) / abs(ref))
            acc[str(2 * n_half)] = {"fds_median": float(np.median(ef)), "fds_max": float(max(ef)),
                                    "fds_plain_accum_median": float(np.median(epl)),
                                    "fds_plain_accum_max": float(max(epl)),
                                    "et_median": float(np.median(ee)), "et_max": float(max(ee))}
        bp = wl.block_diagonal_pair(seed=7, n=20)
        ones = [1] * 40
        tf = _timed(torch, lambda: ctx.lhaf(bp.C, None, ones), reps=3)
        te_ = _timed(torch, lambda: ctx.lhaf(bp.C, None, ones, flags=lg.ET), reps=3)
        out["et_vs_fds"] = {"workload": "block-diagonal A1 (+) A2 of random complex symmetric halves, loops on the "
                                        "diagonal, one photon per index, 5 instances per N",
                            "relative_error_by_N": acc, "fds_ms_N40": tf, "et_ms_N40": te_,
                            "fds_terms_N40": lg.plan(ones)[0], "et_terms_N40": lg.plan(ones, flags=lg.ET)[0]}

    def _grad():
        # adjoint: one 32-photon outcome of a 40-mode state (CUDA events around the host-pointer calls)
        gb = wl.gradient_batch(seed=4, count=2)
        ctx.lhaf_grad(gb.B, gb.gammas[0], gb.reps[0])
        ctx.lhaf(gb.B, gb.gammas[0], gb.reps[0])
        tg = _timed(torch, lambda: ctx.lhaf_grad(gb.B, gb.gammas[0], gb.reps[0]), reps=3)
        tv = _timed(torch, lambda: ctx.lhaf(gb.B, gb.gammas[0], gb.reps[0]), reps=3)
        Tg, ndg, hg, _ = lg.plan(gb.reps[0])
        out["grad"] = {"workload": "value + d/dB + d/dgamma of one 32-photon outcome, 40-mode state",
                       "terms": Tg, "n_dim": ndg, "h": hg, "grad_ms": tg, "value_ms": tv, "grad_over_value": tg / tv}

    def _grad_batch():
        # the differentiated workload: 256 log-probability outcomes of 32 photons (40-mode state),
        # values and gradients from one lhaf_grad_batched call, against the values alone batched
        gb = wl.gradient_batch(seed=4, count=256)
        R = np.stack(gb.reps).astype(np.int32)
        G = np.stack(gb.gammas)
        ctx.lhaf_grad_batched(gb.B, G[:2], R[:2])
        ctx.lhaf_batched(gb.B, G, R)
        tg = _timed(torch, lambda: ctx.lhaf_grad_batched(gb.B, G, R), reps=1)
        tv = _timed(torch, lambda: ctx.lhaf_batched(gb.B, G, R), reps=2)
        vals, _, _, st = ctx.lhaf_grad_batched(gb.B, G[:8], R[:8])
        vb, _ = ctx.lhaf_batched(gb.B, G[:8], R[:8])
        out["grad_batch"] = {"workload": "values and d/dB, d/dgamma of 256 outcomes of 32 photons, 40-mode state",
                             "grad_batched_ms": tg, "values_batched_ms": tv, "grad_over_value": tg / tv,
                             "value_max_rel_diff": float(np.max(np.abs(vals - vb) / np.abs(vb))),
                             "items_ok": int(np.sum(st == 0))}

    steps = (("collision40_and_plain_accum", _collision40_and_plain_accum), ("batched", _batched),
             ("batched_small", _batched_small), ("batched_mode", _batched_mode), ("multi_gamma", _multi_gamma),
             ("chain_rule_step", _chain_rule_step), ("mixed", _mixed), ("et_vs_fds", _et_vs_fds), ("grad", _grad),
             ("grad_batch", _grad_batch))
    for name, f in steps:
        try:
            f()
        except Exception as e:  # one failing extra leaves the rest and the headline
            out.setdefault("extras_errors", {})[name] = repr(e)[:400]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large60", choices=sorted(WORKLOADS))
    ap.add_argument("--terms", type=int, default=None, help="time only the first T terms (profiling runs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    args = ap.parse_args()
    if args.steps < 1 or args.warmup < 0:
        ap.error("--steps must be >= 1 and --warmup >= 0")
    rank, world, local_rank = rank_info()
    if args.gpus != world and world > 1:
        ap.error(f"--gpus {args.gpus} but WORLD_SIZE {world}")
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
