"""Helpers for the GPU parity tests: stores, contexts, oracle references."""
from __future__ import annotations

import os
import tempfile

import numpy as np

import oracle
import synth


def write_both(gs: synth.GraphSet, tmpdir: str | None = None):
    """Write a store file; return (path, oracle.Store)."""
    d = tmpdir or tempfile.mkdtemp(prefix="gcnn_")
    path = os.path.join(d, f"store_{os.getpid()}_{id(gs)}.gcnn")
    synth.write_store(path, gs)
    return path, oracle.read_store(path)


def context(H, L, G, N, E, delta, recompute=False, precision=0, Hh=None, F=0, node_head=0, node_weight=1.0):
    import paper_2207_11333_gb300 as g
    cfg = g.make_config(H, L, G, N, E, delta=delta, recompute=int(recompute), precision=precision,
                        head_hidden=H if Hh is None else Hh, edge_features=F, node_head=node_head,
                        node_loss_weight=node_weight)
    return g.Context(cfg)


def oracle_step(d: oracle.Dims, params_f32, b: oracle.Batch, lr=1e-3):
    """Oracle forward, loss, gradients and one Adam step from float32 parameters."""
    p = params_f32.astype(np.float64)
    loss, grad, _, pred = oracle.backward(d, p, b)
    th = p.copy()
    oracle.adam(th, grad.copy(), np.zeros_like(p), np.zeros_like(p), 1, lr=lr)
    return loss, grad, pred, th
