"""FP64 CPU oracle of the GCNN (PNA) training step -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg import this package.  The library never does.  It shares no
code with the CUDA path; the only common module is ``synth`` (seeded inputs).

The arithmetic is in ``gcnn_oracle.c`` (plain loops, FP64, one function per
step of the method, each citing the paper section it follows).  This file
only marshals numpy arrays and reads the packed store file with its own
reader.

Parity pins (tests/oracle_pins.py, run by tests/test_oracle_pins.py): dense-adjacency matmul for the sum
aggregator, torch.scatter_reduce for all five aggregators, closed forms of the
degree scalers on cycles and stars, node-permutation invariance, pooling of a
constant graph, central finite differences of every gradient, torch autograd
(FP64) on tiny graphs including min/max ties, the first Adam step's closed
form, and numpy lexsort for the collation order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gcnn_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

N_AGG = 5
N_SCALERS = 3


def build(force: bool = False) -> str:
    """Compile gcnn_oracle.c (OpenMP if the compiler has it)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
        try:
            subprocess.check_call(base[:2] + ["-fopenmp"] + base[2:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _SO)
    return _SO


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        _lib = load(_SO)
    return _lib


def load(path: str) -> ctypes.CDLL:
    """Load an oracle shared library and declare its entry points."""
    L = ctypes.CDLL(path)
    i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    L.oracle_collate.restype = i32
    L.oracle_collate.argtypes = [i64, vp, vp, vp, vp, vp, vp, dbl] + [vp] * 11 + [i32, vp, vp, vp, vp]
    L.oracle_delta.restype = dbl
    L.oracle_delta.argtypes = [i64, vp]
    L.oracle_param_count.restype = i64
    L.oracle_param_count.argtypes = [i32, i32, i32, i32, i32, i32]
    L.oracle_forward.restype = i32
    L.oracle_forward.argtypes = [i32, i32, i32, i32, i32, i32, vp, i64, i64, i64] + [vp] * 11 + [dbl, dbl] + [vp] * 5
    L.oracle_backward.restype = i32
    L.oracle_backward.argtypes = [i32, i32, i32, i32, i32, i32, vp, i64, i64, i64] + [vp] * 11 + [dbl, dbl] + [vp] * 6
    L.oracle_adam.restype = None
    L.oracle_adam.argtypes = [i64, vp, vp, vp, vp, i64, dbl, dbl, dbl, dbl, dbl]
    L.oracle_aggregate_op.restype = None
    L.oracle_aggregate_op.argtypes = [i64, i32, vp, vp, dbl, vp]
    L.oracle_aggregate_bwd_op.restype = None
    L.oracle_aggregate_bwd_op.argtypes = [i64, i32, vp, vp, vp, vp, vp]
    return L


def _p(a):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "array must be C-contiguous"
    return a.ctypes.data


# ------------------------------------------------------------------ store

@dataclass
class Store:
    node_ptr: np.ndarray
    edge_ptr: np.ndarray
    types: np.ndarray
    edges: np.ndarray   # uint8 [2E]
    y: np.ndarray
    eattr: np.ndarray | None = None   # float32 [E, F] bond features (version 2 stores)
    ynode: np.ndarray | None = None   # float32 [N] node-level targets (version 2 stores)

    @property
    def F(self) -> int:
        return 0 if self.eattr is None else int(self.eattr.shape[1])


def read_store(path: str) -> Store:
    """Read a packed store file (magic GCNNPKD1, version 1 or 2) into numpy arrays."""
    raw = np.fromfile(path, np.uint8)
    if raw[:8].tobytes() != b"GCNNPKD1":
        raise ValueError("not a packed graph store")
    version = int(raw[8:12].view("<u4")[0])
    G, N, E, o_np, o_ep, o_t, o_e, o_y, size = raw[16:88].view("<i8").tolist()
    if size != raw.size or version not in (1, 2):
        raise ValueError("store size or version mismatch")
    eattr = ynode = None
    if version == 2:
        F, o_a, o_yn = raw[88:112].view("<i8").tolist()
        if F:
            eattr = raw[o_a:o_a + 4 * E * F].view("<f4").reshape(E, F).copy()
        if o_yn:
            ynode = raw[o_yn:o_yn + 4 * N].view("<f4").copy()
    return Store(raw[o_np:o_np + 8 * (G + 1)].view("<i8").copy(),
                 raw[o_ep:o_ep + 8 * (G + 1)].view("<i8").copy(),
                 raw[o_t:o_t + N].copy(),
                 raw[o_e:o_e + 2 * E].copy(),
                 raw[o_y:o_y + 4 * G].view("<f4").copy(), eattr, ynode)


def store_from_arrays(node_ptr, edge_ptr, types, edges, y, eattr=None, ynode=None) -> Store:
    return Store(np.ascontiguousarray(node_ptr, np.int64), np.ascontiguousarray(edge_ptr, np.int64),
                 np.ascontiguousarray(types, np.uint8), np.ascontiguousarray(edges, np.uint8).reshape(-1),
                 np.ascontiguousarray(y, np.float32),
                 None if eattr is None else np.ascontiguousarray(eattr, np.float32),
                 None if ynode is None else np.ascontiguousarray(ynode, np.float32))


# ------------------------------------------------------------------ collation

@dataclass
class Batch:
    G: int
    N: int
    E: int
    node_off: np.ndarray
    edge_off: np.ndarray
    graph_id: np.ndarray
    row_ptr: np.ndarray
    col: np.ndarray
    rev: np.ndarray
    deg: np.ndarray
    amp: np.ndarray
    att: np.ndarray
    types: np.ndarray
    y: np.ndarray
    eattr: np.ndarray   # float32 [E, F] bond features in col order (F = 0: empty)
    ynode: np.ndarray   # float32 [N] node-level targets (zeros when the store has none)

    @property
    def F(self) -> int:
        return int(self.eattr.shape[1])


def collate(st: Store, ids, delta: float) -> Batch:
    """Disjoint union of graphs ``ids`` (oracle_collate)."""
    ids = np.ascontiguousarray(ids, np.int64)
    G = len(ids)
    N = int(np.sum(st.node_ptr[ids + 1] - st.node_ptr[ids]))
    E = int(np.sum(st.edge_ptr[ids + 1] - st.edge_ptr[ids]))
    b = Batch(G, N, E,
              np.zeros(G + 1, np.int64), np.zeros(G + 1, np.int64), np.zeros(N, np.int32),
              np.zeros(N + 1, np.int32), np.zeros(E, np.int32), np.zeros(E, np.int32),
              np.zeros(N, np.int32), np.zeros(N, np.float32), np.zeros(N, np.float32),
              np.zeros(N, np.uint8), np.zeros(G, np.float32), np.zeros((E, st.F), np.float32),
              np.zeros(N, np.float32))
    rc = lib().oracle_collate(G, _p(ids), _p(st.node_ptr), _p(st.edge_ptr), _p(st.types), _p(st.edges),
                              _p(st.y), float(delta), _p(b.node_off), _p(b.edge_off), _p(b.graph_id),
                              _p(b.row_ptr), _p(b.col), _p(b.rev), _p(b.deg), _p(b.amp), _p(b.att),
                              _p(b.types), _p(b.y), st.F, _p(st.eattr), _p(b.eattr), _p(st.ynode), _p(b.ynode))
    if rc:
        raise MemoryError("oracle_collate failed")
    return b


def delta_of(st: Store, ids=None) -> float:
    """delta = mean of log(d+1) over all nodes of the given graphs (default: all)."""
    if ids is None:
        ids = np.arange(len(st.node_ptr) - 1)
    b = collate(st, ids, 1.0)
    return float(lib().oracle_delta(b.N, _p(b.deg)))


# ------------------------------------------------------------------ model

@dataclass
class Dims:
    H: int
    L: int
    T: int = 7
    Hh: int | None = None
    F: int = 0   # bond features per edge
    NH: int = 0  # node-level head (0/1)
    node_weight: float = 1.0  # weight of the node-level MSE in the loss

    def __post_init__(self):
        if self.Hh is None:
            self.Hh = self.H


def param_count(d: Dims) -> int:
    return int(lib().oracle_param_count(d.H, d.L, d.T, d.Hh, d.F, d.NH))


def _batch_args(d: Dims, b: Batch):
    if b.F != d.F:
        raise ValueError(f"batch has {b.F} bond features, the model {d.F}")
    return [b.G, b.N, b.E, _p(b.node_off), _p(b.graph_id), _p(b.row_ptr), _p(b.col), _p(b.deg),
            _p(b.amp), _p(b.att), _p(b.types), _p(b.eattr), _p(b.ynode)]


def forward(d: Dims, params, b: Batch, x0=None, eps: float = 1e-5, want_layers: bool = False,
            want_nodes: bool = False):
    """Predictions (G,) in FP64; with want_layers also xs ((L+1),N,H), aggs (L,N,5H), pooled (G,H);
    with want_nodes (node head) the node-level predictions (N,) are appended."""
    p = np.ascontiguousarray(params, np.float64)
    assert p.size == param_count(d)
    x0a = None if x0 is None else np.ascontiguousarray(x0, np.float64)
    pred = np.zeros(b.G, np.float64)
    xs = np.zeros(((d.L + 1), b.N, d.H)) if want_layers else None
    ag = np.zeros((d.L, b.N, N_AGG * d.H)) if want_layers else None
    pooled = np.zeros((b.G, d.H)) if want_layers else None
    predn = np.zeros(b.N, np.float64) if want_nodes else None
    rc = lib().oracle_forward(d.H, d.L, d.T, d.Hh, d.F, d.NH, _p(p), *_batch_args(d, b), _p(x0a), eps,
                              float(d.node_weight), _p(pred), _p(xs), _p(ag), _p(pooled), _p(predn))
    if rc:
        raise MemoryError("oracle_forward failed")
    out = (pred, xs, ag, pooled) if want_layers else (pred,)
    if want_nodes:
        out = out + (predn,)
    return out if len(out) > 1 else out[0]


def backward(d: Dims, params, b: Batch, x0=None, eps: float = 1e-5, dpred=None):
    """(loss, grad (P,), dx0 (N,H), pred (G,)) in FP64.  Loss is MSE vs b.y unless dpred is given."""
    p = np.ascontiguousarray(params, np.float64)
    x0a = None if x0 is None else np.ascontiguousarray(x0, np.float64)
    dp = None if dpred is None else np.ascontiguousarray(dpred, np.float64)
    grad = np.zeros(p.size, np.float64)
    dx0 = np.zeros((b.N, d.H), np.float64)
    loss = np.zeros(1, np.float64)
    pred = np.zeros(b.G, np.float64)
    rc = lib().oracle_backward(d.H, d.L, d.T, d.Hh, d.F, d.NH, _p(p), *_batch_args(d, b), _p(x0a), eps,
                               float(d.node_weight), _p(b.y), _p(dp),
                               _p(grad), _p(dx0), _p(loss), _p(pred))
    if rc:
        raise MemoryError("oracle_backward failed")
    return float(loss[0]), grad, dx0, pred


def adam(theta, grad, m, v, t: int, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, wd=0.0):
    """In-place AdamW step number t (>= 1) on FP64 arrays."""
    for a in (theta, grad, m, v):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    lib().oracle_adam(theta.size, _p(theta), _p(grad), _p(m), _p(v), t, lr, b1, b2, eps, wd)


# ------------------------------------------------------------------ operators

def aggregate_op(row_ptr, m, eps: float = 1e-5):
    """The aggregation step alone on given per-edge messages m (E, H), slots
    grouped by destination through row_ptr (N+1): (N, 5H) [sum, mean, min,
    max, std] in FP64 (oracle_aggregate_op)."""
    rp = np.ascontiguousarray(row_ptr, np.int32)
    m = np.ascontiguousarray(m, np.float64)
    N, H = rp.size - 1, m.shape[1]
    agg = np.zeros((N, N_AGG * H), np.float64)
    lib().oracle_aggregate_op(N, H, _p(rp), _p(m), eps, _p(agg))
    return agg


def aggregate_bwd_op(row_ptr, m, agg, dagg):
    """dL/dm (E, H) per edge slot from dL/dagg (N, 5H) and the forward's agg
    (oracle_aggregate_bwd_op): min/max ties share, std via (m - mean)/(d std)."""
    rp = np.ascontiguousarray(row_ptr, np.int32)
    m = np.ascontiguousarray(m, np.float64)
    agg = np.ascontiguousarray(agg, np.float64)
    dagg = np.ascontiguousarray(dagg, np.float64)
    N, H = rp.size - 1, m.shape[1]
    assert agg.shape == (N, N_AGG * H) and dagg.shape == (N, N_AGG * H)
    dm = np.zeros_like(m)
    lib().oracle_aggregate_bwd_op(N, H, _p(rp), _p(m), _p(agg), _p(dagg), _p(dm))
    return dm


def split_params(d: Dims, p):
    """Named views of a flat parameter vector (the documented layout)."""
    H, L, T, Hh = d.H, d.L, d.T, d.Hh
    out = {}
    k = 0

    def take(name, shape):
        nonlocal k
        n = int(np.prod(shape))
        out[name] = p[k:k + n].reshape(shape)
        k += n
    take("emb", (T, H))
    for l in range(L):
        take(f"msg_w{l}", (H, 2 * H))
        take(f"msg_b{l}", (H,))
        take(f"upd_w{l}", (16 * H, H))
        take(f"upd_b{l}", (H,))
    take("w1", (H, Hh))
    take("b1", (Hh,))
    take("w2", (Hh,))
    take("b2", (1,))
    if d.F:
        k = (k + 3) // 4 * 4          # bond rows start at a multiple of 4 floats
        for l in range(L):
            take(f"edge_w{l}", (d.F, H))
    if d.NH:
        k = (k + 3) // 4 * 4          # node head likewise
        take("w1n", (H, Hh))
        take("b1n", (Hh,))
        take("w2n", (Hh,))
        take("b2n", (1,))
    assert k == p.size
    return out
