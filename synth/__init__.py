"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

Holds none of the method's arithmetic: graph topology, atom types, random
targets, random parameter vectors, and the packed graph-store file writer.
The generators live in ``synth.c`` (splitmix64 streams + Box-Muller), built
to ``libsynth.so`` beside it.

Packed store file (one file, global arrays; the single-file analogue of the
paper's schema of one global array per graph attribute, Section 4, Table 1):

    offset  type        field
    0       char[8]     magic "GCNNPKD1"
    8       u32         version (1)
    12      u32         number of atom types
    16      i64         G  graphs
    24      i64         N  nodes
    32      i64         E  directed edges
    40      i64         byte offset of node_ptr  (i64[G+1])
    48      i64         byte offset of edge_ptr  (i64[G+1])
    56      i64         byte offset of types     (u8[N])
    64      i64         byte offset of edges     (u8[2E], local (src, dst) pairs)
    72      i64         byte offset of y         (f32[G])
    80      i64         file size in bytes
    88      i64         F  bond features per edge      (version 2 only; may be 0)
    96      i64         byte offset of edge_attr (f32[E][F], version 2, F > 0)
    104     i64         byte offset of node_y    (f32[N], version 2; 0 = none)
    88..127 zero otherwise
Version 2 adds the edges' features (Table 1's edge attributes), one row per
stored directed edge in store order, and node-level targets (Table 1's y at
node level), one per atom.
Every array starts on a 64-byte boundary.  Node and edge ids inside a graph
are local (0..n-1), so a graph is a contiguous slice of each array.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_SO = os.path.join(_HERE, "libsynth.so")
_lib = None

N_TYPES = 7
STORE_MAGIC = b"GCNNPKD1"
HEADER_BYTES = 128


def build(force: bool = False) -> str:
    """Compile synth.c into libsynth.so (plain C, portable flags)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        i64, i32, u64, dbl, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p
        L.synth_stream_first.restype = u64
        L.synth_stream_first.argtypes = [u64, u64, u64]
        L.synth_node_counts.restype = i32
        L.synth_node_counts.argtypes = [u64, i64, i64, i32, i32, i32, dbl, dbl, vp]
        L.synth_max_directed_edges.restype = i64
        L.synth_max_directed_edges.argtypes = [i32, dbl]
        L.synth_topology.restype = i64
        L.synth_topology.argtypes = [u64, i64, i64, vp, i32, dbl, vp, vp, vp, vp, i64]
        L.synth_uniform_targets.restype = None
        L.synth_uniform_targets.argtypes = [u64, i64, i64, dbl, dbl, vp]
        L.synth_normal.restype = None
        L.synth_normal.argtypes = [u64, i64, i64, dbl, vp]
        L.synth_uniform.restype = None
        L.synth_uniform.argtypes = [u64, i64, i64, dbl, dbl, vp]
        L.synth_param_count.restype = i64
        L.synth_param_count.argtypes = [i32, i32, i32, i32]
        L.synth_init_params.restype = None
        L.synth_init_params.argtypes = [u64, i32, i32, i32, i32, vp]
        _lib = L
    return _lib


def _p(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


# ---------------------------------------------------------------- scalars

def node_counts_uniform(seed: int, g0: int, G: int, lo: int, hi: int) -> np.ndarray:
    out = np.empty(G, np.int32)
    rc = lib().synth_node_counts(seed, g0, G, 0, lo, hi, 0.0, 0.0, _p(out))
    if rc:
        raise ValueError(f"synth_node_counts failed ({rc})")
    return out


def node_counts_lognormal(seed: int, g0: int, G: int, mu: float, sigma: float, lo: int, hi: int) -> np.ndarray:
    out = np.empty(G, np.int32)
    rc = lib().synth_node_counts(seed, g0, G, 1, lo, hi, mu, sigma, _p(out))
    if rc:
        raise ValueError(f"synth_node_counts failed ({rc})")
    return out


def lognormal_mu(mean: float = 18.0, sigma: float = 0.45, lo: int = 3, hi: int = 51) -> float:
    """Location mu such that round(exp(N(mu, sigma^2))) truncated to [lo, hi]
    has the requested mean (exact discrete mean, bisection)."""
    def tmean(mu: float) -> float:
        def cdf(x: float) -> float:
            return 0.5 * (1.0 + math.erf((math.log(x) - mu) / (sigma * math.sqrt(2.0))))
        num = den = 0.0
        for k in range(lo, hi + 1):
            p = cdf(k + 0.5) - cdf(max(k - 0.5, 1e-300))
            num += k * p
            den += p
        return num / den
    a, b = math.log(lo), math.log(hi)
    for _ in range(200):
        m = 0.5 * (a + b)
        if tmean(m) < mean:
            a = m
        else:
            b = m
    return 0.5 * (a + b)


def uniform_targets(seed: int, g0: int, G: int, lo: float, hi: float) -> np.ndarray:
    out = np.empty(G, np.float32)
    lib().synth_uniform_targets(seed, g0, G, lo, hi, _p(out))
    return out


def normal(seed: int, i0: int, n: int, sigma: float = 1.0) -> np.ndarray:
    out = np.empty(n, np.float64)
    lib().synth_normal(seed, i0, n, sigma, _p(out))
    return out


def uniform(seed: int, i0: int, n: int, lo: float, hi: float) -> np.ndarray:
    out = np.empty(n, np.float64)
    lib().synth_uniform(seed, i0, n, lo, hi, _p(out))
    return out


def param_count(H: int, L: int, T: int = N_TYPES, Hh: int | None = None, F: int = 0) -> int:
    base = int(lib().synth_param_count(H, L, T, H if Hh is None else Hh))
    return base if F == 0 else (base + 3) // 4 * 4 + L * F * H


def init_params(seed: int, H: int, L: int, T: int = N_TYPES, Hh: int | None = None, F: int = 0) -> np.ndarray:
    """Flat parameters; with F bond features, zero padding up to a multiple of 4
    floats after the head, then the L blocks of bond rows of the message
    weights (F x H each), U(+-1/sqrt(2H + F))."""
    Hh = H if Hh is None else Hh
    base = np.empty(param_count(H, L, T, Hh), np.float32)
    lib().synth_init_params(seed, H, L, T, Hh, _p(base))
    if F == 0:
        return base
    b = 1.0 / math.sqrt(2 * H + F)
    pad = np.zeros((base.size + 3) // 4 * 4 - base.size, np.float32)
    return np.concatenate([base, pad, uniform(seed, 0, L * F * H, -b, b).astype(np.float32)])


# ---------------------------------------------------------------- graphs

@dataclass
class GraphSet:
    """A set of graphs as global arrays (the packed-store layout in memory)."""
    node_ptr: np.ndarray  # int64 [G+1]
    edge_ptr: np.ndarray  # int64 [G+1]
    types: np.ndarray     # uint8 [N]
    edges: np.ndarray     # uint8 [E, 2]  local (src, dst)
    y: np.ndarray         # float32 [G]
    eattr: np.ndarray | None = None   # float32 [E, F] bond features (store version 2)
    ynode: np.ndarray | None = None   # float32 [N] node-level targets (store version 2)

    @property
    def F(self) -> int:
        return 0 if self.eattr is None else int(self.eattr.shape[1])

    @property
    def n_graphs(self) -> int:
        return len(self.node_ptr) - 1

    @property
    def n_nodes(self) -> int:
        return int(self.node_ptr[-1])

    @property
    def n_edges(self) -> int:
        return int(self.edge_ptr[-1])

    def subset(self, ids) -> "GraphSet":
        """Graphs ids[0], ids[1], ... as a new set (local ids are unchanged)."""
        ids = np.asarray(ids, np.int64)
        n = self.node_ptr[ids + 1] - self.node_ptr[ids]
        e = self.edge_ptr[ids + 1] - self.edge_ptr[ids]
        node_ptr = np.zeros(len(ids) + 1, np.int64)
        edge_ptr = np.zeros(len(ids) + 1, np.int64)
        node_ptr[1:] = np.cumsum(n)
        edge_ptr[1:] = np.cumsum(e)
        types = np.concatenate([self.types[self.node_ptr[g]:self.node_ptr[g + 1]] for g in ids]) if len(ids) else np.zeros(0, np.uint8)
        edges = np.concatenate([self.edges[self.edge_ptr[g]:self.edge_ptr[g + 1]] for g in ids]) if len(ids) else np.zeros((0, 2), np.uint8)
        eattr = None
        if self.eattr is not None:
            eattr = (np.concatenate([self.eattr[self.edge_ptr[g]:self.edge_ptr[g + 1]] for g in ids]) if len(ids)
                     else np.zeros((0, self.F), np.float32))
        ynode = None
        if self.ynode is not None:
            ynode = (np.concatenate([self.ynode[self.node_ptr[g]:self.node_ptr[g + 1]] for g in ids]) if len(ids)
                     else np.zeros(0, np.float32))
        return GraphSet(node_ptr, edge_ptr, np.ascontiguousarray(types), np.ascontiguousarray(edges), self.y[ids].copy(),
                        None if eattr is None else np.ascontiguousarray(eattr),
                        None if ynode is None else np.ascontiguousarray(ynode))


def bond_features(seed: int, gs: GraphSet, F: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """F features per bond, U(lo, hi), the same for both stored directions.  The
    generator stores each bond as two consecutive directed edges (u, v), (v, u);
    bond k (0-based over the set) draws items k F .. k F + F - 1."""
    e = gs.edges.reshape(-1, 2)
    if e.shape[0] % 2 or not np.array_equal(e[0::2, 0], e[1::2, 1]) or not np.array_equal(e[0::2, 1], e[1::2, 0]):
        raise ValueError("bond_features: edges are not stored as consecutive (u, v), (v, u) pairs")
    per_bond = uniform(seed, 0, (e.shape[0] // 2) * F, lo, hi).astype(np.float32).reshape(-1, F)
    return np.ascontiguousarray(np.repeat(per_bond, 2, axis=0))


def make_graphs(seed: int, counts: np.ndarray, g0: int = 0, max_deg: int = 4, edge_factor: float = 1.1) -> GraphSet:
    """Topology + atom types for graphs g0.. with the given node counts; y = 0."""
    counts = np.ascontiguousarray(counts, np.int32)
    G = len(counts)
    L = lib()
    # capacity: per-count maximum times multiplicity
    uniq, mult = np.unique(counts, return_counts=True)
    cap = int(sum(int(L.synth_max_directed_edges(int(n), edge_factor)) * int(m) for n, m in zip(uniq, mult)))
    node_ptr = np.zeros(G + 1, np.int64)
    edge_ptr = np.zeros(G + 1, np.int64)
    types = np.zeros(int(counts.sum()), np.uint8)
    edges = np.zeros((max(cap, 1), 2), np.uint8)
    ne = L.synth_topology(seed, g0, G, _p(counts), max_deg, edge_factor, _p(node_ptr), _p(edge_ptr),
                          _p(types), _p(edges), cap)
    if ne < 0:
        raise ValueError(f"synth_topology failed ({ne})")
    return GraphSet(node_ptr, edge_ptr, types, np.ascontiguousarray(edges[:ne]), np.zeros(G, np.float32))


def molecules_uniform(seed: int, G: int, lo: int, hi: int, g0: int = 0) -> GraphSet:
    """G molecule-shaped graphs with n ~ U{lo..hi} nodes (y = 0)."""
    return make_graphs(seed, node_counts_uniform(seed, g0, G, lo, hi), g0=g0)


def molecules_lognormal(seed: int, G: int, mean: float = 18.0, sigma: float = 0.45, lo: int = 3,
                        hi: int = 51, g0: int = 0) -> GraphSet:
    """G molecule-shaped graphs, n = round(exp(N(mu, sigma^2))) in [lo, hi], mu set for the mean."""
    mu = lognormal_mu(mean, sigma, lo, hi)
    return make_graphs(seed, node_counts_lognormal(seed, g0, G, mu, sigma, lo, hi), g0=g0)


# ---------------------------------------------------------------- store file

def _align(x: int, a: int = 64) -> int:
    return (x + a - 1) // a * a


GRAPH_MAGIC = b"GCNNGRF1"


def write_graph_files(directory: str, gs: GraphSet, ids=None) -> list:
    """One file per graph (the layout a packed store replaces); returns the paths.
    Format: magic, int32 n, e, F, float32 y, uint8 types[n], uint8 edges[e][2],
    zero padding to 4 bytes, float32 edge_attr[e][F]."""
    os.makedirs(directory, exist_ok=True)
    paths = []
    for g in (range(gs.n_graphs) if ids is None else ids):
        n0, n1 = int(gs.node_ptr[g]), int(gs.node_ptr[g + 1])
        e0, e1 = int(gs.edge_ptr[g]), int(gs.edge_ptr[g + 1])
        n, e, F = n1 - n0, e1 - e0, gs.F
        head = GRAPH_MAGIC + np.array([n, e, F], "<i4").tobytes() + np.array([gs.y[g]], "<f4").tobytes()
        body = gs.types[n0:n1].tobytes() + np.ascontiguousarray(gs.edges[e0:e1], np.uint8).tobytes()
        pad = b"\0" * ((-(24 + len(body))) % 4)
        attr = np.ascontiguousarray(gs.eattr[e0:e1], "<f4").tobytes() if F else b""
        path = os.path.join(directory, f"g{g:07d}.gcg")
        with open(path, "wb") as f:
            f.write(head + body + pad + attr)
        paths.append(path)
    return paths


def write_store(path: str, gs: GraphSet) -> None:
    """Write a GraphSet as one packed store file (layout in the module docstring)."""
    G, N, E, F = gs.n_graphs, gs.n_nodes, gs.n_edges, gs.F
    v2 = gs.eattr is not None or gs.ynode is not None
    offs = []
    pos = HEADER_BYTES
    sizes = [(G + 1) * 8, (G + 1) * 8, N, 2 * E, 4 * G] + ([4 * E * F] if gs.eattr is not None else [0]) + \
        ([4 * N] if gs.ynode is not None else [0])
    for nbytes in sizes:
        pos = _align(pos)
        offs.append(pos)
        pos += nbytes
    total = _align(pos)
    buf = np.zeros(total, np.uint8)
    hdr = np.zeros(HEADER_BYTES, np.uint8)
    hdr[0:8] = np.frombuffer(STORE_MAGIC, np.uint8)
    hdr[8:16] = np.array([2 if v2 else 1, N_TYPES], "<u4").view(np.uint8)
    hdr[16:88] = np.array([G, N, E] + offs[:5] + [total], "<i8").view(np.uint8)
    if v2:
        hdr[88:112] = np.array([F, offs[5] if F else 0, offs[6] if gs.ynode is not None else 0],
                               "<i8").view(np.uint8)
    buf[:HEADER_BYTES] = hdr
    arrays = [np.ascontiguousarray(gs.node_ptr, "<i8"), np.ascontiguousarray(gs.edge_ptr, "<i8"),
              np.ascontiguousarray(gs.types, np.uint8), np.ascontiguousarray(gs.edges, np.uint8).reshape(-1),
              np.ascontiguousarray(gs.y, "<f4")]
    arrays.append(np.ascontiguousarray(gs.eattr, "<f4").reshape(-1) if gs.eattr is not None
                  else np.zeros(0, np.uint8))
    arrays.append(np.ascontiguousarray(gs.ynode, "<f4") if gs.ynode is not None else np.zeros(0, np.uint8))
    for off, arr in zip(offs, arrays):
        b = arr.view(np.uint8).reshape(-1)
        buf[off:off + b.size] = b
    tmp = path + f".tmp{os.getpid()}"
    buf.tofile(tmp)
    os.replace(tmp, path)
