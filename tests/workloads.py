"""Seeded workloads used by the tests (sizes follow the configurations they stand for).

small_parity(): 64 graphs of 5-30 nodes, H = 32, L = 2, 2-layer head 32->32->1,
targets = a fixed seeded teacher of the same architecture (FP64 oracle) plus
N(0, 0.05^2) noise.  Seeds: data 1, teacher 2, student 3, noise 4.
"""
from __future__ import annotations

import numpy as np

import oracle
import synth

SEED_DATA, SEED_TEACHER, SEED_STUDENT, SEED_NOISE = 1, 2, 3, 4


def small_parity(G: int = 64, lo: int = 5, hi: int = 30, H: int = 32, L: int = 2):
    d = oracle.Dims(H=H, L=L)
    gs = synth.molecules_uniform(SEED_DATA, G, lo, hi)
    st = oracle.store_from_arrays(gs.node_ptr, gs.edge_ptr, gs.types, gs.edges, gs.y)
    delta = oracle.delta_of(st)
    b = oracle.collate(st, np.arange(G), delta)
    teacher = synth.init_params(SEED_TEACHER, H, L).astype(np.float64)
    y = oracle.forward(d, teacher, b) + synth.normal(SEED_NOISE, 0, G, 0.05)
    gs.y = y.astype(np.float32)
    student = synth.init_params(SEED_STUDENT, H, L)
    return d, gs, delta, student
