"""Writes chain_rule_ill_conditioned.json: extended-precision values of the most ill-conditioned
loop hafnians of the 4096-item chain-rule batch (seeded generator, 50-mode lossy state), from
the C oracle's long double build through repeated matrix products (the route whose per-term
rounding is smallest: Newton's identities amplify the characteristic polynomial's), with each
sum's condition number (sum |weight * f| / |sum|) and the FP64 C oracle's value beside it.
Calls only oracle/ (and the seeded input generator). Run from the repository root:
    python tests/golden/make_chain_rule_ill_conditioned.py"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import csieve  # noqa: E402
from paper_2108_01622_gb300 import workloads as wl  # noqa: E402

# the items whose sums cancel the most (found by comparing two FP64 evaluations of the batch)
ITEMS = (2684, 1484, 3039)


def main():
    b = wl.chain_rule_batch(seed=3, count=4096)
    items = []
    for i in ITEMS:
        reps = np.asarray(b.reps[i], dtype=np.int32)
        g = b.gammas[i]
        ext, mag, _ = csieve._sieve(b.B, g, reps, 0, None, False, 0, True)
        h = (int(reps.sum()) + 1) // 2
        val = ext / 2 ** h
        fp64 = csieve.lhaf(b.B, g, reps)
        items.append({"index": int(i), "photons": int(reps.sum()),
                      "value": [float(np.real(val)), float(np.imag(val))],
                      "value_lo": [float(np.real(val) - np.longdouble(float(np.real(val)))),
                                   float(np.imag(val) - np.longdouble(float(np.imag(val))))],
                      "condition": mag / float(abs(ext)),
                      "fp64_c_oracle": [fp64.real, fp64.imag]})
        print(items[-1], flush=True)
    out = {"source": "oracle/lhaf_sieve.c built with LHAF_ORACLE_EXTENDED (long double), repeated products; "
                     "workloads.chain_rule_batch(seed=3, count=4096)",
           "items": items}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "chain_rule_ill_conditioned.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
