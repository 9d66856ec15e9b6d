"""Run a few loop hafnians of one named workload through the C ABI (device inputs), for profiler
captures of the sieve kernels:  python -m paper_2108_01622_gb300.profile_case <workload> [calls]

workloads: single24 (24 photons, collision-free), collision40 (40 photons over 22 modes),
large60_slice (2^16 terms of the 60-photon collision-free sum)."""
import sys

import numpy as np


def main():
    import torch

    import paper_2108_01622_gb300 as lg
    from paper_2108_01622_gb300 import workloads as wl

    name = sys.argv[1] if len(sys.argv) > 1 else "collision40"
    calls = int(sys.argv[2]) if len(sys.argv) > 2 else 2
    flags = 0
    if name == "single24":
        p = wl.single_lhaf_24(seed=1)
    elif name == "collision40":
        p = wl.collision_lhaf_40(seed=2)
        flags = lg.NO_LOOPS
    elif name == "large60_slice":
        p = wl.large_lhaf_60(seed=5)
    else:
        raise SystemExit(f"unknown workload {name}")
    dev = torch.device("cuda", 0)
    with lg.Context(0) as ctx:
        Bd = torch.from_numpy(p.B).to(dev)
        gd = torch.from_numpy(p.gamma).to(dev)
        for _ in range(calls):
            if name == "large60_slice":
                r, st = ctx.lhaf_range(Bd, gd, p.reps, 0, 1 << 16, stats=True)
            else:
                r, st = ctx.lhaf(Bd, gd, p.reps, flags=flags, stats=True)
            torch.cuda.synchronize()
            print(name, st, flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
