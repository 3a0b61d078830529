"""Writes small_parity_oracle.txt: FP64 oracle results on the 64-graph parity workload.

Calls only synth (seeded inputs) and oracle/.  Run from the repository root:
    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path[:0] = [ROOT, os.path.join(ROOT, "tests")]

import oracle  # noqa: E402
import workloads  # noqa: E402


def main():
    d, gs, delta, student = workloads.small_parity()
    st = oracle.store_from_arrays(gs.node_ptr, gs.edge_ptr, gs.types, gs.edges, gs.y)
    b = oracle.collate(st, np.arange(gs.n_graphs), delta)
    p = student.astype(np.float64)
    loss, grad, _, pred = oracle.backward(d, p, b)
    views = oracle.split_params(d, grad)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "small_parity_oracle.txt")
    with open(out, "w") as f:
        f.write("# FP64 oracle on the 64-graph parity workload (tests/workloads.py: small_parity)\n")
        f.write("# written by tests/golden/make_golden.py; values: delta, loss, pred[0..63], |grad| per tensor\n")
        f.write(f"delta {delta:.17g}\n")
        f.write(f"loss {loss:.17g}\n")
        for g, v in enumerate(pred):
            f.write(f"pred {g} {v:.17g}\n")
        for k, v in views.items():
            f.write(f"gradnorm {k} {np.linalg.norm(v):.17g}\n")


if __name__ == "__main__":
    main()
