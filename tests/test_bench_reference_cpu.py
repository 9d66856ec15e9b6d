"""bench.py's reference arm runs the oracle as it stands on the host cores (no GPU): its JSON line
carries the contract's keys, and the same metric, unit and workload as the GPU arm."""
import json
import os
import subprocess
import sys


def test_reference_arm_json_line():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["config"]["workload"].startswith("60-photon collision-free loop hafnian")
    assert line["config"]["evaluated_terms"] == 2 ** 29


def test_bench_rank_step_ranges_cover_the_sum_once():
    # N > 1: each rank takes its share of the terms of the one loop hafnian, cut into the steps;
    # together the ranges tile [0, T) in term order (the all-gather concatenates them rank by rank)
    from tests.libutil import ensure_built

    ensure_built()
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    for T, world, steps in ((2 ** 29, 1, 20), (2 ** 29, 2, 20), (1000, 3, 7), (5, 4, 3), (2 ** 20, 8, 5)):
        flat = [r for rank in range(world) for r in bench.rank_step_ranges(T, rank, world, steps)]
        assert len(flat) == world * steps
        assert flat[0][0] == 0 and flat[-1][1] == T
        assert all(a[1] == b[0] for a, b in zip(flat, flat[1:]))
        assert all(b >= a for a, b in flat)
