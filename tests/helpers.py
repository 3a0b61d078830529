"""Shared test fixtures: seeded graph sets, oracle batches, error measures."""
from __future__ import annotations

import math

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


def star_and_dense_set(seed: int = 41, ks=(5, 8, 16, 64, 254), dense: int = 6, max_deg: int = 16):
    """Stars K_{1,k} (centre in-degree k, leaves 1; leaf types cycle over the 7
    atom types, so the centre sees groups of equal messages: ties) followed by
    `dense` molecule-shaped graphs of 20-60 atoms with degrees up to max_deg
    (2.5 bonds per atom, so many atoms have more than 4 neighbours).  Every
    graph stays within the store's limits (255 atoms, 1,024 directed edges)."""
    graphs = [([1] + [j % 7 for j in range(k)], [(0, j) for j in range(1, k + 1)]) for k in ks]
    stars = custom_set(graphs)
    if not dense:
        return stars
    mol = synth.make_graphs(seed, synth.node_counts_uniform(seed, 0, dense, 20, 60), max_deg=max_deg,
                            edge_factor=2.5)
    t = [(stars.types[stars.node_ptr[g]:stars.node_ptr[g + 1]].tolist(),
          [tuple(e) for e in stars.edges[stars.edge_ptr[g]:stars.edge_ptr[g + 1]:2].tolist()])
         for g in range(stars.n_graphs)]
    t += [(mol.types[mol.node_ptr[g]:mol.node_ptr[g + 1]].tolist(),
           [tuple(e) for e in mol.edges[mol.edge_ptr[g]:mol.edge_ptr[g + 1]:2].tolist()])
          for g in range(mol.n_graphs)]
    return custom_set(t)


# Gates of the parity tests (relative errors: normwise, and elementwise below)
FP32_FWD_TOL = 1e-5     # FP32 forward: predictions and every layer's activations
FP32_GRAD_TOL = 1e-4    # FP32 gradients: every parameter tensor
BF16_FWD_TOL = 2e-2     # BF16-GEMM forward, normwise
BF16_U = 2.0 ** -8      # unit roundoff of bfloat16 (8 significant bits, round to nearest)


def bf16_fwd_bound(L: int) -> float:
    """First-order forward error of the BF16-GEMM path: every BF16 GEMM rounds
    both operands once (relative error <= u each, FP32 accumulation adds
    K 2^-24 <= 2e-4, negligible), so one GEMM output carries <= 2u; a forward
    pass chains 2 GEMMs per layer (message, update) and the errors add:
    2u * 2L."""
    return 2 * BF16_U * 2 * L


def bf16_grad_bound(L: int, kappa: float = 1.0) -> float:
    """Normwise bound for a parameter gradient of the BF16-GEMM path against the
    FP64 oracle, from two error sources (neither taken from a measurement):

    rounding along the path: <= 2u per BF16 GEMM output, at most 4L + 1 of
      them between the loss and a weight gradient (2L forward, 2 per layer
      of the backward above the tensor, the weight-gradient GEMM itself),
      amplified by kappa = ||yhat|| / ||yhat - y|| (>= 1) because the loss
      gradient is the residual yhat - y;
    decisions: the ReLU masks and the min/max routes are decided on forward
      values that carry <= e = bf16_fwd_bound(L) relative error; an entry
      whose margin is below e can flip, which with margins of density <= 1
      near 0 is a fraction <= e of the entries, and a flip moves at most the
      entry's own gradient (twice its square in the norm): sqrt(2 e).
    """
    return 2 * BF16_U * (4 * L + 1) * max(1.0, kappa) + math.sqrt(2 * bf16_fwd_bound(L))


def residual_kappa(pred, y) -> float:
    """kappa = ||yhat|| / ||yhat - y|| (at least 1) from the oracle's predictions."""
    pred = np.asarray(pred, np.float64)
    r = np.linalg.norm(pred - np.asarray(y, np.float64))
    return max(1.0, float(np.linalg.norm(pred) / r)) if r > 0 else float("inf")


def rel_max_rms(a, b) -> float:
    """max |a - b| / max(|b|, rms(b)) elementwise: the largest error of any entry,
    relative to that entry or, for entries below it, to the tensor's RMS."""
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    if b.size == 0:
        return 0.0
    floor = max(float(np.sqrt(np.mean(b * b))), 1e-300)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), floor)))


# Elementwise gate = ELEM_FACTOR x the normwise gate, on rel_max_rms.  Rounding
# errors of a correct FP32 (or BF16) computation are spread over a tensor's n
# entries; their largest is about sqrt(2 ln n) <= 5.3 times their RMS for
# n <= 10^6 (Gaussian tail), and their RMS relative to the tensor's RMS is the
# normwise error: the factor 10 leaves a margin of 2.  An error confined to a
# few entries (one wrong row of a rare node class) is not diluted by sqrt(n)
# here, as it is in the norm.  R13's own elementwise measure, floored at 1e-3
# of the largest entry, is reported beside it: it gives an entry at that floor
# an absolute budget of 1e-8 (forward) of the largest entry, below the rounding
# of the K = 16H products that form it, so no FP32 implementation meets it.
ELEM_FACTOR = 10.0


class Gates:
    """Collects relative errors of many tensors, prints them all, and fails
    once at the end with every tensor that broke its gate.

    check(name, a, b, tol): normwise rel_norm < tol and, unless
    elementwise=False, rel_max_rms < ELEM_FACTOR * tol; R13's rel_max is
    printed for reference.  A reference that is exactly zero must be matched
    exactly."""

    def __init__(self, title: str):
        self.title = title
        self.rows = []

    def check(self, name, a, b, tol: float, elementwise: bool = True):
        b64 = np.asarray(b, np.float64)
        if b64.size and np.max(np.abs(b64)) == 0.0:
            en = float(np.max(np.abs(np.asarray(a, np.float64))))     # an exactly-zero reference
            self.rows.append((name, en, en, float("nan"), tol, None, en <= 0.0))
            return
        en = rel_norm(a, b)
        ee = rel_max_rms(a, b) if elementwise else float("nan")
        r13 = rel_max(a, b)
        et = ELEM_FACTOR * tol if elementwise else None
        ok = en < tol and (et is None or ee < et)
        self.rows.append((name, en, ee, r13, tol, et, ok))

    def check_abs(self, name, err, scale, tol: float):
        """Componentwise: max |err| / scale < tol, with scale the magnitude of
        the operands that formed each entry (FP32 error analysis)."""
        err = np.abs(np.asarray(err, np.float64)).ravel()
        scale = np.asarray(scale, np.float64).ravel()
        with np.errstate(divide="ignore", invalid="ignore"):
            q = np.where(scale > 0, err / np.where(scale > 0, scale, 1.0), np.where(err > 0, np.inf, 0.0))
        m = float(np.max(q)) if q.size else 0.0
        self.rows.append((name, float("nan"), m, float("nan"), None, tol, m < tol))

    def report(self) -> str:
        lines = [f"{self.title}: tensor, normwise, elementwise (rms floor), R13 rel_max, gates"]
        for name, en, ee, r13, nt, et, ok in self.rows:
            gates = (f"<{nt:.0e}" if nt else "") + (f" <{et:.0e}" if et else "")
            lines.append(f"  {name:14s} {en:9.2e} {ee:9.2e} {r13:9.2e}  {gates}" + ("" if ok else "  FAIL"))
        return "\n".join(lines)

    def assert_all(self):
        text = self.report()
        print(text)
        bad = [r[0] for r in self.rows if not r[6]]
        assert not bad, f"gates broken by {bad}\n{text}"
