"""Python binding of libgcnn (include/gcnn.h): argument marshalling only.

Every step of the GCNN training / inference path runs in the library's CUDA
kernels; this module converts numpy arrays / torch tensors to pointers,
passes torch's current CUDA stream, and turns status codes into exceptions.
There is no fallback: if libgcnn.so is missing or cannot be loaded, importing
this package raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgcnn.so")

PREC_FP32 = 0
PREC_BF16 = 1
FLAG_ROW_INVARIANT = 1
FLAG_SERIAL = 2
PHASES = ["collate", "embed", "gemm", "agg_fwd", "agg_bwd", "head", "embed_bwd", "adam"]
NPHASE = len(PHASES)
# kernel identifiers of the timeline records (GCNN_K_* in gcnn.h)
KERNELS = {1: "collate_scan", 2: "collate_graph", 3: "embed", 4: "embed_bwd", 5: "agg_fwd", 6: "agg_bwd_edge",
           7: "agg_bwd_gather", 8: "gemm_tc_partial", 9: "gemm_tc_c", 10: "gemm_tc_d3", 11: "gemm_tc_reduce",
           12: "gemm_simt", 13: "gemm_simt_reduce", 14: "pool_fwd", 15: "pool_bwd", 16: "head_graph",
           17: "head_grad", 18: "colsum", 19: "adam", 20: "cast_bf16", 21: "pack_layer", 22: "step_end",
           23: "agg_bwd_fused", 24: "agg_bwd_chunks", 25: "node_pred", 26: "node_grad", 27: "bond_grad",
           28: "collate"}

_ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "EFORMAT", -5: "EDEVICE", -6: "ETIMEDOUT",
           -7: "EAGAIN", -8: "ESTATE"}


class GcnnError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRORS.get(code, code)}: {msg}")
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [("hidden", ctypes.c_int32), ("layers", ctypes.c_int32), ("n_types", ctypes.c_int32),
                ("head_hidden", ctypes.c_int32), ("max_graphs", ctypes.c_int32), ("max_nodes", ctypes.c_int32),
                ("max_edges", ctypes.c_int32), ("precision", ctypes.c_int32), ("recompute", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("delta", ctypes.c_double), ("std_eps", ctypes.c_double),
                ("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("adam_eps", ctypes.c_double),
                ("weight_decay", ctypes.c_double), ("edge_features", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("node_head", ctypes.c_int32), ("reserved1", ctypes.c_int32), ("node_loss_weight", ctypes.c_double)]


class BatchStruct(ctypes.Structure):
    _fields_ = [("n_graphs", ctypes.c_int32), ("n_nodes", ctypes.c_int32), ("n_edges", ctypes.c_int32),
                ("reserved", ctypes.c_int32)] + [(n, ctypes.c_void_p) for n in (
                    "node_off", "edge_off", "graph_id", "row_ptr", "col", "rev", "deg", "amp", "att", "types", "y",
                    "edge_attr", "node_y")]


class ServeConfig(ctypes.Structure):
    _fields_ = [("n_slots", ctypes.c_int32), ("n_buckets", ctypes.c_int32), ("bucket_nodes", ctypes.c_int32 * 8),
                ("max_graphs", ctypes.c_int32), ("precision", ctypes.c_int32), ("queue_nodes", ctypes.c_int64)]


class RequestStruct(ctypes.Structure):
    _fields_ = [("n_mol", ctypes.c_int32), ("reserved", ctypes.c_int32), ("n_nodes", ctypes.c_void_p),
                ("n_edges", ctypes.c_void_p), ("types", ctypes.c_void_p), ("edges", ctypes.c_void_p)]


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run paper_2207_11333_gb300.build.build() "
                          "(there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    i32, i64, f32, f64, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double, ctypes.c_void_p
    P = ctypes.POINTER
    sig = {
        "gcnn_last_error": (ctypes.c_char_p, []),
        "gcnn_version": (i32, []),
        "gcnn_store_open": (i32, [ctypes.c_char_p, P(vp)]),
        "gcnn_store_close": (i32, [vp]),
        "gcnn_store_info": (i32, [vp, P(i64), P(i64), P(i64)]),
        "gcnn_store_edge_features": (i32, [vp, P(i32)]),
        "gcnn_store_has_node_targets": (i32, [vp, P(i32)]),
        "gcnn_get_node_predictions": (i32, [vp, vp, i64]),
        "gcnn_store_pack": (i32, [vp, i64, ctypes.c_char_p, i32]),
        "gcnn_collate_files": (i32, [vp, vp, i32, vp]),
        "gcnn_store_batch_size": (i32, [vp, vp, i64, P(i64), P(i64)]),
        "gcnn_store_delta": (i32, [vp, vp, i64, P(f64)]),
        "gcnn_store_set_targets": (i32, [vp, vp, i64]),
        "gcnn_store_to_device": (i32, [vp]),
        "gcnn_config_default": (i32, [P(Config), i32, i32, i32, i32, i32]),
        "gcnn_create": (i32, [P(Config), vp, P(vp)]),
        "gcnn_destroy": (i32, [vp]),
        "gcnn_param_count": (i32, [vp, P(i64)]),
        "gcnn_set_params": (i32, [vp, vp, i64, i32]),
        "gcnn_get_params": (i32, [vp, vp, i64, i32]),
        "gcnn_get_grads": (i32, [vp, vp, i64, i32]),
        "gcnn_reset_optimizer": (i32, [vp]),
        "gcnn_save": (i32, [vp, ctypes.c_char_p]),
        "gcnn_load": (i32, [vp, ctypes.c_char_p]),
        "gcnn_check": (i32, [vp]),
        "gcnn_collate": (i32, [vp, vp, vp, i32, P(BatchStruct)]),
        "gcnn_set_order": (i32, [vp, vp, vp, i64]),
        "gcnn_collate_range": (i32, [vp, vp, i64, i32, P(BatchStruct)]),
        "gcnn_batch_export": (i32, [vp, P(BatchStruct)] + [vp] * 10),
        "gcnn_forward": (i32, [vp, P(BatchStruct), vp, i32]),
        "gcnn_backward": (i32, [vp, P(BatchStruct), vp, vp]),
        "gcnn_step": (i32, [vp, f32]),
        "gcnn_set_loss_scale": (i32, [vp, f32, f32]),
        "gcnn_grad_buckets": (i32, [vp, P(i32)]),
        "gcnn_grad_bucket": (i32, [vp, i32, P(i64), P(i64)]),
        "gcnn_grad_wait": (i32, [vp, i32, vp]),
        "gcnn_grads_device": (i32, [vp, P(vp)]),
        "gcnn_train_step": (i32, [vp, P(BatchStruct), f32, vp]),
        "gcnn_train_step_range": (i32, [vp, vp, i64, i32, f32, vp, P(BatchStruct)]),
        "gcnn_forward_backward": (i32, [vp, P(BatchStruct), vp]),
        "gcnn_get_activation": (i32, [vp, i32, vp, i64]),
        "gcnn_profile_enable": (i32, [vp, i32]),
        "gcnn_profile_read": (i32, [vp, vp, vp]),
        "gcnn_step_kernel_count": (i32, [vp, P(i32)]),
        "gcnn_timeline_enable": (i32, [vp, i32]),
        "gcnn_ffma_peak": (i32, [i32, P(f64)]),
        "gcnn_gemm_study": (i32, [i32, i32, i32, vp, i32, P(i32)]),
        "gcnn_timeline_read": (i32, [vp, vp, vp, i32, P(i32)]),
        "gcnn_memory": (i32, [vp, P(i64)]),
        "gcnn_serve_create": (i32, [vp, P(ServeConfig), P(vp)]),
        "gcnn_serve_submit": (i32, [vp, P(RequestStruct), P(ctypes.c_uint64)]),
        "gcnn_serve_poll": (i32, [vp, ctypes.c_uint64, vp, P(f64)]),
        "gcnn_serve_wait": (i32, [vp, ctypes.c_uint64, vp, P(f64), i64]),
        "gcnn_serve_stats": (i32, [vp, P(i64), P(i64), P(i64), P(i64)]),
        "gcnn_serve_destroy": (i32, [vp]),
        "gcnn_serve_timing": (i32, [vp, P(f64), P(f64), P(f64), P(i64)]),
        "gcnn_op_aggregate_fwd": (i32, [i32, i32, vp, vp, vp, vp, f32, vp]),
        "gcnn_op_aggregate_bwd": (i32, [i32, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, f32, vp]),
        "gcnn_op_aggregate_bwd_graphs": (i32, [i32, i32, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, f32, vp]),
        "gcnn_op_aggregate_bwd_noalloc": (i32, [i32, i32, i32, vp, vp, vp, vp, vp, vp, vp, f32, vp]),
        "gcnn_op_pool_fwd": (i32, [i32, i32, vp, vp, vp, vp]),
        "gcnn_op_pool_bwd": (i32, [i32, i32, i32, vp, vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


lib = _load()


def _check(rc: int) -> None:
    if rc != 0:
        raise GcnnError(rc, lib.gcnn_last_error().decode(errors="replace"))


def _np_ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "array must be C-contiguous"
    return a.ctypes.data


def _stream(stream=None):
    """cudaStream_t of torch's current stream (or the given torch stream / raw handle)."""
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_ptr(t, dtype=None):
    """Device pointer of a contiguous CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


# ---------------------------------------------------------------- store

def _c_paths(paths):
    arr = (ctypes.c_char_p * max(len(paths), 1))()
    for k, p in enumerate(paths):
        arr[k] = os.fsencode(p)
    return arr


def store_pack(paths, out_path: str, n_threads: int = 1) -> None:
    """Pack per-graph files (gcnn_store_pack) into one store file."""
    arr = _c_paths(paths)
    _check(lib.gcnn_store_pack(ctypes.cast(arr, ctypes.c_void_p), len(paths), os.fsencode(out_path), int(n_threads)))


class Store:
    """Packed graph store (gcnn_store_*)."""

    def __init__(self, path: str):
        self._h = ctypes.c_void_p()
        _check(lib.gcnn_store_open(path.encode(), ctypes.byref(self._h)))
        g, n, e = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib.gcnn_store_info(self._h, ctypes.byref(g), ctypes.byref(n), ctypes.byref(e)))
        self.n_graphs, self.n_nodes, self.n_edges = g.value, n.value, e.value
        f = ctypes.c_int32()
        _check(lib.gcnn_store_edge_features(self._h, ctypes.byref(f)))
        self.edge_features = f.value
        _check(lib.gcnn_store_has_node_targets(self._h, ctypes.byref(f)))
        self.has_node_targets = bool(f.value)

    @property
    def handle(self):
        return self._h

    def close(self) -> None:
        if self._h:
            _check(lib.gcnn_store_close(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def batch_size(self, ids) -> tuple[int, int]:
        ids = np.ascontiguousarray(ids, np.int64)
        n, e = ctypes.c_int64(), ctypes.c_int64()
        _check(lib.gcnn_store_batch_size(self._h, _np_ptr(ids), len(ids), ctypes.byref(n), ctypes.byref(e)))
        return n.value, e.value

    def delta(self, ids=None) -> float:
        d = ctypes.c_double()
        if ids is None:
            _check(lib.gcnn_store_delta(self._h, None, 0, ctypes.byref(d)))
        else:
            ids = np.ascontiguousarray(ids, np.int64)
            _check(lib.gcnn_store_delta(self._h, _np_ptr(ids), len(ids), ctypes.byref(d)))
        return d.value

    def set_targets(self, y) -> None:
        y = np.ascontiguousarray(y, np.float32)
        _check(lib.gcnn_store_set_targets(self._h, _np_ptr(y), len(y)))

    def to_device(self) -> None:
        _check(lib.gcnn_store_to_device(self._h))


# ---------------------------------------------------------------- context

def ffma_peak(iters: int = 4096) -> float:
    """FP32 FFMA throughput of the current device, TFLOP/s (measurement support)."""
    t = ctypes.c_double()
    _check(lib.gcnn_ffma_peak(int(iters), ctypes.byref(t)))
    return t.value


GEMM_SHAPES = ("message", "update", "dW_U", "dagg", "dW_M", "dx")


def gemm_study(n_atoms: int, hidden: int, mode: int = 0, max_rows: int = 4096) -> list[dict]:
    """Timing study of the training step's BF16 GEMMs (gcnn_gemm_study): one dict per timed plan."""
    rows = np.zeros((max_rows, 8), np.float64)
    n = ctypes.c_int32()
    _check(lib.gcnn_gemm_study(int(n_atoms), int(hidden), int(mode), _np_ptr(rows), max_rows, ctypes.byref(n)))
    return [{"shape": GEMM_SHAPES[int(r[0])], "BN": int(r[1]), "ntiles": int(r[2]), "splits": int(r[3]),
             "cluster": bool(r[4]), "K": int(r[5]), "us": float(r[6]), "planner": bool(r[7])} for r in rows[:n.value]]


def make_config(hidden: int, layers: int, max_graphs: int, max_nodes: int, max_edges: int, **kw) -> Config:
    c = Config()
    _check(lib.gcnn_config_default(ctypes.byref(c), hidden, layers, max_graphs, max_nodes, max_edges))
    for k, v in kw.items():
        if not hasattr(c, k):
            raise AttributeError(k)
        setattr(c, k, v)
    return c


@dataclass
class Batch:
    s: BatchStruct
    owner: "Context"

    @property
    def n_graphs(self) -> int:
        return self.s.n_graphs

    @property
    def n_nodes(self) -> int:
        return self.s.n_nodes

    @property
    def n_edges(self) -> int:
        return self.s.n_edges

    def export(self) -> dict:
        G, N, E = self.n_graphs, self.n_nodes, self.n_edges
        out = {"node_off": np.zeros(G + 1, np.int32), "graph_id": np.zeros(N, np.int32),
               "row_ptr": np.zeros(N + 1, np.int32), "col": np.zeros(E, np.int32), "rev": np.zeros(E, np.int32),
               "deg": np.zeros(N, np.int32), "amp": np.zeros(N, np.float32), "att": np.zeros(N, np.float32),
               "types": np.zeros(N, np.uint8), "y": np.zeros(G, np.float32)}
        _check(lib.gcnn_batch_export(self.owner._h, ctypes.byref(self.s), *[_np_ptr(out[k]) for k in (
            "node_off", "graph_id", "row_ptr", "col", "rev", "deg", "amp", "att", "types", "y")]))
        return out

    def tensor(self, name: str):
        """A torch view of one of the batch's device arrays (valid until the next collate)."""
        import torch
        G, N, E = self.n_graphs, self.n_nodes, self.n_edges
        if name == "edge_attr":  # E rows of round_up(F, 4) floats; the first F columns hold the features
            F = self.owner.cfg.edge_features
            F4 = (F + 3) // 4 * 4
            return _wrap_device(self.s.edge_attr, E * F4, torch.float32).view(E, F4)[:, :F]
        spec = {"node_off": (G + 1, torch.int32), "edge_off": (G + 1, torch.int32), "graph_id": (N, torch.int32),
                "row_ptr": (N + 1, torch.int32), "col": (E, torch.int32), "rev": (E, torch.int32),
                "deg": (N, torch.int32), "amp": (N, torch.float32), "att": (N, torch.float32),
                "types": (N, torch.uint8), "y": (G, torch.float32), "node_y": (N, torch.float32)}[name]
        return _wrap_device(getattr(self.s, name), spec[0], spec[1])


def _wrap_device(ptr: int, n: int, dtype):
    """Zero-copy torch tensor over library-owned device memory (via DLPack-free __cuda_array_interface__)."""
    import torch
    typestr = {torch.int32: "<i4", torch.float32: "<f4", torch.uint8: "|u1", torch.int64: "<i8"}[dtype]

    class _A:
        __cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr or 0, False), "version": 2}
    if n == 0:
        return torch.zeros(0, dtype=dtype, device="cuda")
    return torch.as_tensor(_A(), device="cuda")


class Context:
    """A training context (gcnn_create): parameters, Adam state, activation arena."""

    def __init__(self, cfg: Config, stream=None):
        self.cfg = cfg
        self._h = ctypes.c_void_p()
        _check(lib.gcnn_create(ctypes.byref(cfg), _stream(stream), ctypes.byref(self._h)))
        n = ctypes.c_int64()
        _check(lib.gcnn_param_count(self._h, ctypes.byref(n)))
        self.n_params = n.value

    def close(self) -> None:
        if self._h:
            _check(lib.gcnn_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # parameters
    def set_params(self, p) -> None:
        if isinstance(p, np.ndarray):
            p = np.ascontiguousarray(p, np.float32)
            _check(lib.gcnn_set_params(self._h, _np_ptr(p), p.size, 0))
        else:
            _check(lib.gcnn_set_params(self._h, _dev_ptr(p, None), p.numel(), 1))

    def get_params(self) -> np.ndarray:
        out = np.empty(self.n_params, np.float32)
        _check(lib.gcnn_get_params(self._h, _np_ptr(out), out.size, 0))
        return out

    def get_grads(self) -> np.ndarray:
        out = np.empty(self.n_params, np.float32)
        _check(lib.gcnn_get_grads(self._h, _np_ptr(out), out.size, 0))
        return out

    def reset_optimizer(self) -> None:
        _check(lib.gcnn_reset_optimizer(self._h))

    # data parallelism (Sec. 4): hooks for an exchange of the gradients
    def set_loss_scale(self, graph_scale: float, node_scale: float = 1.0) -> None:
        _check(lib.gcnn_set_loss_scale(self._h, float(graph_scale), float(node_scale)))

    def grad_buckets(self) -> list[tuple[int, int]]:
        """(offset, count) of every gradient bucket: layers 0..L-1, head (+ bond
        rows, node head), embedding."""
        n = ctypes.c_int32()
        _check(lib.gcnn_grad_buckets(self._h, ctypes.byref(n)))
        out = []
        for k in range(n.value):
            o, c = ctypes.c_int64(), ctypes.c_int64()
            _check(lib.gcnn_grad_bucket(self._h, k, ctypes.byref(o), ctypes.byref(c)))
            out.append((o.value, c.value))
        return out

    def grad_wait(self, bucket: int, stream) -> None:
        """Order `stream` (torch stream or raw handle) after bucket's final gradients."""
        _check(lib.gcnn_grad_wait(self._h, int(bucket), _stream(stream)))

    def grads_tensor(self):
        """Zero-copy torch view of the flat FP32 gradient buffer on the device."""
        import torch
        p = ctypes.c_void_p()
        _check(lib.gcnn_grads_device(self._h, ctypes.byref(p)))
        return _wrap_device(p.value, self.n_params, torch.float32)

    def save(self, path: str) -> None:
        _check(lib.gcnn_save(self._h, path.encode()))

    def load(self, path: str) -> None:
        _check(lib.gcnn_load(self._h, path.encode()))

    def check(self) -> None:
        _check(lib.gcnn_check(self._h))

    # batches
    def collate(self, store: Store, ids) -> Batch:
        ids = np.ascontiguousarray(ids, np.int64)
        b = BatchStruct()
        _check(lib.gcnn_collate(self._h, store.handle, _np_ptr(ids), len(ids), ctypes.byref(b)))
        return Batch(b, self)

    def collate_files(self, paths) -> Batch:
        """Collate graphs straight from per-graph files (gcnn_collate_files)."""
        arr = _c_paths(paths)
        b = BatchStruct()
        _check(lib.gcnn_collate_files(self._h, ctypes.cast(arr, ctypes.c_void_p), len(paths), ctypes.byref(b)))
        return Batch(b, self)

    def set_order(self, store: Store, order) -> None:
        order = np.ascontiguousarray(order, np.int64)
        _check(lib.gcnn_set_order(self._h, store.handle, _np_ptr(order), len(order)))

    def collate_range(self, store: Store, first: int, count: int) -> Batch:
        b = BatchStruct()
        _check(lib.gcnn_collate_range(self._h, store.handle, first, count, ctypes.byref(b)))
        return Batch(b, self)

    # training
    def forward(self, batch: Batch, pred=None, train: bool = True) -> None:
        _check(lib.gcnn_forward(self._h, ctypes.byref(batch.s), _dev_ptr(pred), int(train)))

    def backward(self, batch: Batch, dpred=None, loss_accum=None) -> None:
        _check(lib.gcnn_backward(self._h, ctypes.byref(batch.s), _dev_ptr(dpred), _dev_ptr(loss_accum)))

    def step(self, lr: float) -> None:
        _check(lib.gcnn_step(self._h, lr))

    def train_step(self, batch: Batch, lr: float, loss_accum=None) -> None:
        _check(lib.gcnn_train_step(self._h, ctypes.byref(batch.s), lr, _dev_ptr(loss_accum)))

    def train_step_range(self, store: Store, first: int, count: int, lr: float, loss_accum=None) -> Batch:
        """Collation of order[first:first+count] and one training step in one graph (gcnn_train_step_range)."""
        b = BatchStruct()
        _check(lib.gcnn_train_step_range(self._h, store.handle, first, count, lr, _dev_ptr(loss_accum),
                                         ctypes.byref(b)))
        return Batch(b, self)

    def forward_backward(self, batch: Batch, loss_accum=None) -> None:
        """Captured forward + backward without the optimizer (gcnn_forward_backward)."""
        _check(lib.gcnn_forward_backward(self._h, ctypes.byref(batch.s), _dev_ptr(loss_accum)))

    def profile(self, enable: bool) -> None:
        _check(lib.gcnn_profile_enable(self._h, int(enable)))

    def profile_read(self) -> dict:
        ms = np.zeros(NPHASE, np.float64)
        n = np.zeros(NPHASE, np.int64)
        _check(lib.gcnn_profile_read(self._h, _np_ptr(ms), _np_ptr(n)))
        return {name: (float(ms[i]), int(n[i])) for i, name in enumerate(PHASES)}

    def timeline_enable(self, capacity: int) -> None:
        """Record (kernel id, device ns) at the start of every library kernel; 0 disables."""
        _check(lib.gcnn_timeline_enable(self._h, int(capacity)))

    def timeline_read(self, max_records: int = 1 << 16):
        """Records since the last read: (kernel ids int32[n], device times in ns int64[n])."""
        ids = np.zeros(max_records, np.int32)
        t = np.zeros(max_records, np.int64)
        n = ctypes.c_int32()
        _check(lib.gcnn_timeline_read(self._h, _np_ptr(ids), _np_ptr(t), int(max_records), ctypes.byref(n)))
        return ids[:n.value].copy(), t[:n.value].copy()

    def memory_bytes(self) -> int:
        n = ctypes.c_int64()
        _check(lib.gcnn_memory(self._h, ctypes.byref(n)))
        return n.value

    def step_kernel_count(self) -> int:
        k = ctypes.c_int32()
        _check(lib.gcnn_step_kernel_count(self._h, ctypes.byref(k)))
        return k.value

    def activation(self, layer: int) -> np.ndarray:
        n = self._last_nodes * self.cfg.hidden
        out = np.empty(n, np.float32)
        _check(lib.gcnn_get_activation(self._h, layer, _np_ptr(out), n))
        return out.reshape(self._last_nodes, self.cfg.hidden)

    def activations(self, batch: Batch) -> list[np.ndarray]:
        self._last_nodes = batch.n_nodes
        return [self.activation(l) for l in range(self.cfg.layers + 1)]

    def node_predictions(self, batch: Batch) -> np.ndarray:
        """Node-level outputs of the last forward (node head), N floats."""
        out = np.empty(batch.n_nodes, np.float32)
        _check(lib.gcnn_get_node_predictions(self._h, _np_ptr(out), batch.n_nodes))
        return out


# ---------------------------------------------------------------- operators

def aggregate_fwd(PQ, row_ptr, col, std_eps: float = 1e-5, stream=None):
    """agg (N x 5H) = [sum, mean, min, max, std] of P_i + Q_j over each CSR row (gcnn_op_aggregate_fwd)."""
    import torch
    N, H2 = PQ.shape
    H = H2 // 2
    agg = torch.empty(N, 5 * H, device=PQ.device, dtype=torch.float32)
    _check(lib.gcnn_op_aggregate_fwd(N, H, _dev_ptr(row_ptr, torch.int32), _dev_ptr(col, torch.int32),
                                     _dev_ptr(PQ, torch.float32), _dev_ptr(agg), std_eps, _stream(stream)))
    return agg


def aggregate_bwd(PQ, agg, dagg, row_ptr, col, rev, std_eps: float = 1e-5, stream=None, node_off=None):
    """dPQ (N x 2H) from dagg: gcnn_op_aggregate_bwd, or gcnn_op_aggregate_bwd_graphs
    when the graph offsets node_off (G + 1 int32) are given."""
    import torch
    N, H2 = PQ.shape
    H = H2 // 2
    E = col.numel()
    dPQ = torch.empty_like(PQ)
    ptrs = (_dev_ptr(row_ptr, torch.int32), _dev_ptr(col, torch.int32), _dev_ptr(rev, torch.int32),
            _dev_ptr(PQ, torch.float32), _dev_ptr(agg, torch.float32), _dev_ptr(dagg.contiguous(), torch.float32),
            _dev_ptr(dPQ))
    if node_off is None:
        scratch = torch.empty(max(E, 1) * H, device=PQ.device, dtype=torch.float32)
        _check(lib.gcnn_op_aggregate_bwd(N, E, H, *ptrs, _dev_ptr(scratch), std_eps, _stream(stream)))
    else:
        scratch = torch.empty(E * H + E + 2, device=PQ.device, dtype=torch.float32)
        _check(lib.gcnn_op_aggregate_bwd_graphs(node_off.numel() - 1, N, E, H, _dev_ptr(node_off, torch.int32),
                                                *ptrs, _dev_ptr(scratch), std_eps, _stream(stream)))
    return dPQ


def pool_fwd(x, node_off, stream=None):
    import torch
    G = node_off.numel() - 1
    H = x.shape[1]
    out = torch.empty(G, H, device=x.device, dtype=torch.float32)
    _check(lib.gcnn_op_pool_fwd(G, H, _dev_ptr(node_off, torch.int32), _dev_ptr(x, torch.float32), _dev_ptr(out),
                                _stream(stream)))
    return out


def pool_bwd(dpooled, node_off, graph_id, n_nodes: int, stream=None):
    import torch
    G, H = dpooled.shape
    dx = torch.empty(n_nodes, H, device=dpooled.device, dtype=torch.float32)
    _check(lib.gcnn_op_pool_bwd(G, n_nodes, H, _dev_ptr(node_off, torch.int32), _dev_ptr(graph_id, torch.int32),
                                _dev_ptr(dpooled.contiguous(), torch.float32), _dev_ptr(dx), _stream(stream)))
    return dx


# ---------------------------------------------------------------- serving

class Server:
    """Continuous-batching inference server (gcnn_serve_*) over a trained Context."""

    def __init__(self, model: Context, n_slots: int = 4, buckets=(1024, 4096, 16384, 65536), max_graphs: int = 4096,
                 precision: int = PREC_FP32, queue_nodes: int = 1 << 22):
        cfg = ServeConfig()
        cfg.n_slots, cfg.n_buckets, cfg.max_graphs = n_slots, len(buckets), max_graphs
        for i, b in enumerate(buckets):
            cfg.bucket_nodes[i] = b
        cfg.precision, cfg.queue_nodes = precision, queue_nodes
        self._h = ctypes.c_void_p()
        _check(lib.gcnn_serve_create(model._h, ctypes.byref(cfg), ctypes.byref(self._h)))
        self._n = {}

    def submit(self, n_nodes, n_edges, types, edges):
        """Queue one request; returns a ticket, or None when admission is refused (queue full)."""
        nn = np.ascontiguousarray(n_nodes, np.int32)
        ne = np.ascontiguousarray(n_edges, np.int32)
        ty = np.ascontiguousarray(types, np.uint8)
        ed = np.ascontiguousarray(edges, np.uint8).reshape(-1)
        q = RequestStruct(len(nn), 0, _np_ptr(nn), _np_ptr(ne), _np_ptr(ty), _np_ptr(ed) if ed.size else _np_ptr(ty))
        t = ctypes.c_uint64()
        rc = lib.gcnn_serve_submit(self._h, ctypes.byref(q), ctypes.byref(t))
        if rc == -7:
            return None
        _check(rc)
        self._n[t.value] = len(nn)
        return t.value

    def poll(self, ticket: int):
        """(predictions, latency_us) when done, else None."""
        out = np.empty(self._n[ticket], np.float32)
        lat = ctypes.c_double()
        rc = lib.gcnn_serve_poll(self._h, ticket, _np_ptr(out), ctypes.byref(lat))
        if rc == -7:
            return None
        del self._n[ticket]
        _check(rc)
        return out, lat.value

    def wait(self, ticket: int, timeout_s: float = 60.0):
        out = np.empty(self._n[ticket], np.float32)
        lat = ctypes.c_double()
        rc = lib.gcnn_serve_wait(self._h, ticket, _np_ptr(out), ctypes.byref(lat), int(timeout_s * 1e6))
        if rc != -6:
            del self._n[ticket]
        _check(rc)
        return out, lat.value

    def stats(self) -> dict:
        v = [ctypes.c_int64() for _ in range(4)]
        _check(lib.gcnn_serve_stats(self._h, *[ctypes.byref(x) for x in v]))
        return dict(zip(("requests", "molecules", "batches", "refused"), (x.value for x in v)))

    def timing(self) -> dict:
        """Host scheduler time, device time and atoms summed over batches (gcnn_serve_timing)."""
        h, d, a, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
        _check(lib.gcnn_serve_timing(self._h, ctypes.byref(h), ctypes.byref(d), ctypes.byref(a), ctypes.byref(n)))
        return {"host_us": h.value, "device_us": d.value, "atoms": a.value, "batches": n.value}

    def close(self) -> None:
        if self._h:
            _check(lib.gcnn_serve_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def request_arrays(gs, first: int, count: int):
    """(n_nodes, n_edges, types, edges) of graphs first..first+count-1 of a synth.GraphSet."""
    a, b = gs.node_ptr[first], gs.node_ptr[first + count]
    c, d = gs.edge_ptr[first], gs.edge_ptr[first + count]
    return (np.diff(gs.node_ptr[first:first + count + 1]).astype(np.int32),
            np.diff(gs.edge_ptr[first:first + count + 1]).astype(np.int32), gs.types[a:b], gs.edges[c:d])
