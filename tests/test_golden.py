"""The oracle reproduces its stored results on the parity workload (regression pin, no GPU).

tests/golden/small_parity_oracle.txt was written by tests/golden/make_golden.py,
which calls only synth and oracle/.  A later change to the oracle's arithmetic
must come with a regenerated file and a reason.
"""
import os

import numpy as np

import oracle
import workloads
from helpers import rel_norm

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "small_parity_oracle.txt")


def _read():
    vals = {"pred": {}, "gradnorm": {}}
    for line in open(GOLDEN):
        if line.startswith("#"):
            continue
        f = line.split()
        if f[0] in ("pred", "gradnorm"):
            vals[f[0]][f[1]] = float(f[2])
        else:
            vals[f[0]] = float(f[1])
    return vals


def test_oracle_matches_golden():
    g = _read()
    d, gs, delta, student = workloads.small_parity()
    assert abs(delta - g["delta"]) <= 1e-14 * g["delta"]
    st = oracle.store_from_arrays(gs.node_ptr, gs.edge_ptr, gs.types, gs.edges, gs.y)
    b = oracle.collate(st, np.arange(gs.n_graphs), delta)
    loss, grad, _, pred = oracle.backward(d, student.astype(np.float64), b)
    assert abs(loss - g["loss"]) <= 1e-11 * g["loss"]
    assert rel_norm(pred, [g["pred"][str(i)] for i in range(len(pred))]) < 1e-12
    for k, v in oracle.split_params(d, grad).items():
        assert abs(np.linalg.norm(v) - g["gradnorm"][k]) <= 1e-10 * g["gradnorm"][k], k
