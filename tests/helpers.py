"""Shared test fixtures: seeded graph sets, oracle batches, error measures."""
from __future__ import annotations

import numpy as np

import oracle
import synth


def rel_norm(a, b) -> float:
    """Normwise relative error ||a - b|| / ||b||."""
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def rel_max(a, b) -> float:
    """max |a - b| / max(|b|, 1e-3 ||b||_inf) elementwise."""
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    if b.size == 0:
        return 0.0
    floor = max(1e-3 * float(np.max(np.abs(b))), 1e-300)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), floor)))


def graph_set(seed: int, G: int, lo: int, hi: int, y_seed: int | None = 99) -> synth.GraphSet:
    gs = synth.molecules_uniform(seed, G, lo, hi)
    if y_seed is not None:
        gs.y = synth.uniform_targets(y_seed, 0, G, 1.0, 10.0)
    return gs


def to_store(gs: synth.GraphSet) -> oracle.Store:
    return oracle.store_from_arrays(gs.node_ptr, gs.edge_ptr, gs.types, gs.edges, gs.y, gs.eattr, gs.ynode)


def oracle_batch(gs: synth.GraphSet, ids=None, delta: float | None = None):
    st = to_store(gs)
    if ids is None:
        ids = np.arange(gs.n_graphs)
    if delta is None:
        delta = oracle.delta_of(st)
    return st, oracle.collate(st, ids, delta), delta


def custom_set(graphs) -> synth.GraphSet:
    """GraphSet from a list of (types, undirected edge list) pairs; each edge stored both ways."""
    node_ptr, edge_ptr, types, edges = [0], [0], [], []
    for t, und in graphs:
        types.extend(t)
        for u, v in und:
            edges.append((u, v))
            edges.append((v, u))
        node_ptr.append(node_ptr[-1] + len(t))
        edge_ptr.append(edge_ptr[-1] + 2 * len(und))
    return synth.GraphSet(np.array(node_ptr, np.int64), np.array(edge_ptr, np.int64),
                          np.array(types, np.uint8), np.array(edges, np.uint8).reshape(-1, 2),
                          np.zeros(len(graphs), np.float32))
