"""Test helpers: make sure the in-tree CUDA library exists (building it with nvcc if needed)."""
import os

import paper_2108_01622_gb300 as lg


def ensure_built():
    if not os.path.exists(lg.LIB_PATH):
        from paper_2108_01622_gb300 import build

        build.build()
    return lg
