"""Throughput of the loop-hafnian sieve on GB300 (one JSON line on rank 0).

Step = one loop hafnian of the collision-pattern workload (100-mode Haar kernel, 40 photons over 22
modes with counts 1..4, gamma = 0, complex128): host pairing plan, slot-matrix gather, every sieve
term on the GPU, double-double reduction. Inputs are resident on the device when the timed region
starts; the L2 is flushed (256 MiB write) between timed steps, outside the per-step events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun, one rank per GPU: every rank evaluates its own loop hafnian (independent
problems, no data-path collective; weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "lhaf sieve terms/s (collision-pattern loop hafnian, FP64)"
UNIT = "terms/s"
WORKLOAD = ("collision-pattern loop hafnian: 100-mode Haar interferometer, r ~ U[1.0,1.6], gamma = 0, "
            "40 photons over 22 modes with counts 1..4 (seeded multinomial), complex128, repeated-pair sieve")
KERNEL_NAME = "grouped_terms_kernel (FP64 sieve terms of the zero-digit groups)"
# DRAM bytes (read + write) of one grouped_terms_kernel launch on this workload, from the ncu
# capture summarised in profiles/grouped_terms_kernel_collision40.md (None once the kernel changes)
KERNEL_TRAFFIC_BYTES = 221696
NOMINAL_FP64_GFLOPS = 152 * 4 * 0.5 * 2 * 2.070  # SMs x sub-partitions x FMA lanes/clk x 2 flops x GHz


def rank_info():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


# ------------------------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm): the oracle as it stands, on a bounded
# sample of the same workload's sieve terms, spread over the host cores with a spawn pool.
# ------------------------------------------------------------------------------------------


def _oracle_slice(args):
    seed, start, stop = args
    sys.path.insert(0, ROOT)
    from oracle import lhaf_oracle as lo
    from paper_2108_01622_gb300 import workloads as wl

    p = wl.collision_lhaf_40(seed=seed)
    t0 = time.perf_counter()
    terms = lo.repeated_sieve_terms(p.B, p.gamma, p.reps, start, stop)
    return len(terms), time.perf_counter() - t0


class OracleTimer:
    """The oracle as it stands, timed on slices of the workload's sieve terms over all host cores
    (one spawn pool, created before any GPU call)."""

    def __init__(self):
        import multiprocessing as mp

        from oracle import lhaf_oracle as lo
        from paper_2108_01622_gb300 import workloads as wl

        p = wl.collision_lhaf_40(seed=2)
        self.total_terms = lo.repeated_term_count(p.reps)
        self.cores = os.cpu_count() or 1
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:  # one BLAS thread per worker process: `cores` is the number of processes
            os.environ[k] = "1"
        self.pool = mp.get_context("spawn").Pool(self.cores)
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
        self.pool.map(_oracle_slice, [(2, 0, 64)] * self.cores)  # workers import numpy, warm up
        n, dt = _oracle_slice((2, 0, 256))
        self.per_term = dt / max(n, 1)
        self.cursor = 256

    def sample(self, seconds: float):
        per_worker = max(64, int(seconds / self.per_term))
        chunks = []
        for _ in range(self.cores):
            if self.cursor + per_worker > self.total_terms:
                self.cursor = 0
            chunks.append((2, self.cursor, self.cursor + per_worker))
            self.cursor += per_worker
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_slice, chunks)
        wall = time.perf_counter() - t0
        done = sum(r[0] for r in res)
        rate = done / wall
        return {"value": rate, "unit": UNIT, "cores": self.cores, "kind": "oracle",
                "sample": f"{done} sieve terms (slices of the {self.total_terms}-term unhalved sum of the same "
                          f"workload), numpy oracle, {self.cores}-process spawn pool, {wall:.1f} s wall",
                "ms_per_lhaf": self.total_terms / rate * 1e3, "terms_per_lhaf": self.total_terms}

    def close(self):
        self.pool.close()
        self.pool.join()


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------

CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, index: int, path: str):
        self.path = path
        self.proc = None
        try:
            self.f = open(path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={CLOCK_FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
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


# ------------------------------------------------------------------------------------------


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    timer = OracleTimer()
    per_step = min(10.0, max(0.3, 150.0 / (args.steps + args.warmup)))
    rates = []
    base = None
    for s in range(args.warmup + args.steps):
        r = timer.sample(per_step)
        if s >= args.warmup:
            rates.append(r["value"])
        base = r
    timer.close()
    value = statistics.median(rates)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": base["ms_per_lhaf"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": base["cores"], "kind": "oracle",
                             "sample": base["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, rank, world, local_rank):
    import torch

    import paper_2108_01622_gb300 as lg
    from paper_2108_01622_gb300 import workloads as wl

    cpu_base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        timer = OracleTimer()  # spawn pool started before the first GPU call
        cpu_base = timer.sample(15.0)
        timer.close()

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    p = wl.collision_lhaf_40(seed=2)
    T, nd, h, P = lg.plan(p.reps, has_loops=False)
    groups = lg.plan_groups(p.reps, has_loops=False)
    ctx = lg.Context(local_rank)  # ordered on torch's current stream
    Bd = torch.from_numpy(p.B).to(dev)
    gd = torch.from_numpy(p.gamma).to(dev)
    flags = lg.NO_LOOPS
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    fp64_gflops = lg.fp64_probe(local_rank)

    out = torch.empty(1, dtype=torch.complex128, device=dev)
    for _ in range(args.warmup):
        ctx.lhaf(Bd, gd, p.reps, flags=flags, out=out)
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kern_ms = []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank, os.path.join(ROOT, "gpurun_out", f"clocks_rank{rank}.csv")
                           if os.path.isdir(os.path.join(ROOT, "gpurun_out")) else f"/tmp/clocks_rank{rank}.csv")
    time.sleep(0.3)
    stats = None
    launches = 0
    for s in range(args.steps):
        flush.zero_()
        starts[s].record()
        _, stats = ctx.lhaf(Bd, gd, p.reps, flags=flags, out=out, stats=True)
        ends[s].record()
        kern_ms.append(stats["kernel_ms"])
        launches += stats["launches"]
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * args.steps * T / (total_ms * 1e-3)
    val = complex(out.cpu()[0])

    # e2e: the public host-pointer call (pinned staging copies inside the library) per step
    _, est = ctx.lhaf(p.B, p.gamma, p.reps, stats=True)  # bytes the host path copies per call
    e2e_times = []
    for s in range(max(3, args.steps // 4)):
        t0 = time.perf_counter()
        ctx.lhaf(p.B, p.gamma, p.reps)
        e2e_times.append(time.perf_counter() - t0)
    e2e_ms = statistics.median(e2e_times) * 1e3

    extras = {} if args.no_extras else run_extras(ctx, torch, dev, lg, wl)

    avg_kernel_ms = statistics.mean(kern_ms)
    flops = stats["flops_model"]
    achieved = flops / (avg_kernel_ms * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "terms_per_lhaf": T, "n_dim": nd, "h": h, "pairs": P,
                   "team": stats["team"], "zero_digit_groups": groups,
                   "l2": "flushed between steps (256 MiB write, outside step events)",
                   "parallelism": f"{world} independent loop hafnians, one per GPU"},
        "ms_per_lhaf": total_ms / args.steps,
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "kernel": KERNEL_NAME if groups else "terms_kernel (FP64 sieve terms)",
                     "achieved": achieved, "peak": NOMINAL_FP64_GFLOPS / 1e3, "unit": "TFLOP/s",
                     "frac": achieved / (NOMINAL_FP64_GFLOPS / 1e3),
                     "traffic": KERNEL_TRAFFIC_BYTES if groups else None,
                     "peak_source": "derived: 152 SMs x 4 sub-partitions x 0.5 FP64 FMA lanes/clk x 2 x 2.070 GHz",
                     "fp64_probe_tflops": fp64_gflops / 1e3,
                     "frac_of_probe": achieved / (fp64_gflops / 1e3),
                     "flops_per_launch": flops, "avg_launch_ms": avg_kernel_ms},
        "e2e": {"value": T / (e2e_ms * 1e-3), "unit": UNIT, "ms_per_lhaf": e2e_ms,
                "h2d_bytes_per_step": est["h2d_bytes"], "d2h_bytes_per_step": est["d2h_bytes"]},
        "clocks": clocks,
        "result": [val.real, val.imag],
    }
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
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    return statistics.median(times)


def run_extras(ctx, torch, dev, lg, wl):
    """The rest of the metric, each on its own workload (untimed by the step loop above):
    ms per 60-photon loop hafnian (projected from a timed slice of its sieve terms), the FP32-term
    variant on the same slice, batched vs one call per item on a chain-rule batch, the batched mode of
    one chain-rule step, a mixed-state probability, and the adjoint."""
    out = {}
    # 60-photon collision-free lhaf (100-mode Haar, r ~ U[1.2, 1.8]): 2^29 terms of dimension 61
    p60 = wl.large_lhaf_60(seed=5)
    T60, nd60, h60, _ = lg.plan(p60.reps)
    B60 = torch.from_numpy(p60.B).to(dev)
    g60 = torch.from_numpy(p60.gamma).to(dev)
    S = 1 << 17
    ctx.lhaf_range(B60, g60, p60.reps, 0, 4096)  # tunes the team size for this shape
    ms64 = _timed(torch, lambda: ctx.lhaf_range(B60, g60, p60.reps, 0, S), reps=2)
    ctx.lhaf_range(B60, g60, p60.reps, 0, 4096, flags=lg.FP32_TERMS)
    ms32 = _timed(torch, lambda: ctx.lhaf_range(B60, g60, p60.reps, 0, S, flags=lg.FP32_TERMS), reps=2)
    msp = _timed(torch, lambda: ctx.lhaf_range(B60, g60, p60.reps, 0, S, flags=lg.PLAIN_ACCUM), reps=2)
    pd = ctx.lhaf_range(p60.B, p60.gamma, p60.reps, 0, S)
    pp = ctx.lhaf_range(p60.B, p60.gamma, p60.reps, 0, S, flags=lg.PLAIN_ACCUM)
    sd, sp = complex(pd[0] + pd[1], pd[2] + pd[3]), complex(pp[0] + pp[1], pp[2] + pp[3])
    fl = lg.flops_per_term(nd60, h60, True)
    out["lhaf60"] = {"workload": "60-photon collision-free loop hafnian, 100-mode Haar, r~U[1.2,1.8], complex gamma",
                     "terms_per_lhaf": T60, "n_dim": nd60, "h": h60, "timed_terms": S,
                     "ms_per_60_photon_lhaf_projected": ms64 * T60 / S, "fp64_tflops": fl * S / (ms64 * 1e-3) / 1e12,
                     "fp32_terms_ms_per_lhaf_projected": ms32 * T60 / S, "fp32_speedup": ms64 / ms32,
                     "plain_accum_ms_per_lhaf_projected": msp * T60 / S,
                     "plain_vs_dd_slice_rel_diff": abs(sp - sd) / abs(sd),
                     "note": "projected = timed slice x (terms / slice); every term costs the same"}
    # batched vs one call per item: 512 loop hafnians of the chain-rule batch (N in 10..40)
    b = wl.chain_rule_batch(seed=3, count=512)
    R = np.array(b.reps)
    Gd = torch.from_numpy(np.array(b.gammas)).to(dev)
    Bd = torch.from_numpy(b.B).to(dev)
    ob = torch.empty(len(R), dtype=torch.complex128, device=dev)
    op = torch.empty(len(R), dtype=torch.complex128, device=dev)
    ctx.lhaf_batched(Bd, Gd, R, out=ob)
    for i in range(len(R)):  # warm the per-shape tuning cache of the single-call path
        ctx.lhaf(Bd, Gd[i], R[i], out=op[i:i + 1])
    torch.cuda.synchronize()
    tb = _timed(torch, lambda: ctx.lhaf_batched(Bd, Gd, R, out=ob), reps=2)

    def plain():
        for i in range(len(R)):
            ctx.lhaf(Bd, Gd[i], R[i], out=op[i:i + 1])

    tp = _timed(torch, plain, reps=2)
    d = (ob - op).abs() / op.abs()
    og = torch.empty(len(R), dtype=torch.complex128, device=dev)
    with ctx.batched_plan(Bd, Gd, R) as plan:
        plan.run(Bd, Gd, out=og)
        tg_ = _timed(torch, lambda: plan.run(Bd, Gd, out=og), reps=2)
    dg = (og - op).abs() / op.abs()
    out["batched"] = {"workload": "chain-rule batch: 512 loop hafnians, 50-mode lossy GBS state, N~U{10..40}",
                      "batched_ms": tb, "graph_replay_ms": tg_, "plain_ms": tp,
                      "batched_over_plain_speedup": tp / tb, "graph_over_plain_speedup": tp / tg_,
                      "max_rel_diff": float(max(d.max().item(), dg.max().item()))}
    # small items only: many short loop hafnians, where one launch per item is launch-bound
    bs = wl.chain_rule_batch(seed=7, count=2048, n_lo=8, n_hi=16)
    Rs = np.array(bs.reps)
    Gs = torch.from_numpy(np.array(bs.gammas)).to(dev)
    Bs = torch.from_numpy(bs.B).to(dev)
    obs = torch.empty(len(Rs), dtype=torch.complex128, device=dev)
    ops_ = torch.empty(len(Rs), dtype=torch.complex128, device=dev)
    ctx.lhaf_batched(Bs, Gs, Rs, out=obs)
    for i in range(len(Rs)):
        ctx.lhaf(Bs, Gs[i], Rs[i], out=ops_[i:i + 1])
    tbs = _timed(torch, lambda: ctx.lhaf_batched(Bs, Gs, Rs, out=obs), reps=2)

    def plain_s():
        for i in range(len(Rs)):
            ctx.lhaf(Bs, Gs[i], Rs[i], out=ops_[i:i + 1])

    tps = _timed(torch, plain_s, reps=2)
    ogs = torch.empty(len(Rs), dtype=torch.complex128, device=dev)
    with ctx.batched_plan(Bs, Gs, Rs) as plan:
        plan.run(Bs, Gs, out=ogs)
        tgs = _timed(torch, lambda: plan.run(Bs, Gs, out=ogs), reps=3)
    out["batched_small"] = {"workload": "2048 loop hafnians, N~U{8..16}, same state family",
                            "batched_ms": tbs, "graph_replay_ms": tgs, "plain_ms": tps,
                            "batched_over_plain_speedup": tps / tbs, "graph_over_plain_speedup": tps / tgs}
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
    ctx.lhaf(cb.B, gm, pats[-1])
    tl = _timed(torch, lambda: ctx.lhaf(cb.B, gm, pats[-1]), reps=3)
    vm = ctx.lhaf_batched_mode(cb.B, gm, fixed, mode, n_cut)
    vb, _ = ctx.lhaf_batched(cb.B, gms, pats)
    out["batched_mode"] = {"workload": f"chain-rule step: {int(fixed.sum())} fixed photons, outcomes 0..{n_cut} "
                                       "of the next mode, 50-mode lossy state",
                           "batched_mode_ms": tm, "batched_patterns_ms": tbp, "speedup": tbp / tm,
                           "largest_outcome_alone_ms": tl, "batched_mode_over_largest": tm / tl,
                           "max_rel_diff": float(np.max(np.abs(vm - vb) / np.abs(vb)))}
    # several loop-weight vectors on one pattern (App. B.5, threshold sub-detectors): 16 vectors on
    # the 40-photon collision pattern, against the same 16 loop hafnians as one batch
    pm_ = wl.collision_lhaf_40(seed=2)
    Gm = wl.complex_normal(np.random.default_rng(21), (16, len(pm_.reps)))
    Rm = np.repeat(np.asarray(pm_.reps)[None, :], 16, axis=0)
    vm_ = ctx.lhaf_multi_gamma(pm_.B, Gm, pm_.reps)
    vb_, _ = ctx.lhaf_batched(pm_.B, Gm, Rm)
    tmg = _timed(torch, lambda: ctx.lhaf_multi_gamma(pm_.B, Gm, pm_.reps), reps=3)
    tbg = _timed(torch, lambda: ctx.lhaf_batched(pm_.B, Gm, Rm), reps=3)
    out["multi_gamma"] = {"workload": "16 loop-weight vectors on the 40-photon collision pattern (100-mode Haar)",
                          "multi_gamma_ms": tmg, "batched_ms": tbg, "speedup": tbg / tmg,
                          "max_rel_diff": float(np.max(np.abs(vm_ - vb_) / np.abs(vb_)))}
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
    # mixed state (App. B.2 lhafmix): a 20-photon outcome of a 50-mode lossy state, the loop
    # hafnian of the 100 x 100 matrix A with every occupied index pair repeated
    ms_ = wl.lossy_state(seed=12, M=50, r_lo=0.8, r_hi=1.4, eta=0.6)
    nm = wl.pattern_multinomial(np.random.default_rng(12), 50, 20, 3)
    Tm, ndm, hm, _ = lg.plan(np.concatenate([nm, nm]))
    ctx.gbs_pattern_prob_mixed(ms_.sigma, ms_.alpha, nm)
    tmx = _timed(torch, lambda: ctx.gbs_pattern_prob_mixed(ms_.sigma, ms_.alpha, nm), reps=3)
    out["mixed"] = {"workload": "P(n) of a 20-photon outcome (counts <= 3) of a 50-mode lossy state, eta = 0.6",
                    "terms": Tm, "n_dim": ndm, "h": hm, "ms": tmx}
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
    # adjoint: one 32-photon outcome of a 40-mode state
    gb = wl.gradient_batch(seed=4, count=2)
    import time as _t
    ctx.lhaf_grad(gb.B, gb.gammas[0], gb.reps[0])
    t0 = _t.perf_counter()
    ctx.lhaf_grad(gb.B, gb.gammas[0], gb.reps[0])
    tg = (_t.perf_counter() - t0) * 1e3
    t0 = _t.perf_counter()
    ctx.lhaf(gb.B, gb.gammas[0], gb.reps[0])
    tv = (_t.perf_counter() - t0) * 1e3
    Tg, ndg, hg, _ = lg.plan(gb.reps[0])
    out["grad"] = {"workload": "value + d/dB + d/dgamma of one 32-photon outcome, 40-mode state",
                   "terms": Tg, "n_dim": ndg, "h": hg, "grad_ms": tg, "value_ms": tv, "grad_over_value": tg / tv}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    args = ap.parse_args()
    rank, world, local_rank = rank_info()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
