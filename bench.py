#!/usr/bin/env python
"""Training throughput of the GCNN (PNA) step on GB300, graphs/s.

Workload (synthetic stand-in for PCQM4Mv2 / AISD, which are not available):
200,000 molecule-shaped graphs (3-51 nodes, truncated log-normal with mean
18, mean degree 2.2, max degree 4, 7 atom types), 6 PNA layers of width 200,
head 200 -> 200 -> 1, batch 128 graphs, AdamW lr 1e-3, targets from a seeded
teacher of the same architecture mapped to [1, 10] eV.  One step = collate +
forward + backward + optimizer over one batch.

`value`: device time of K steps (CUDA events per step on the launching
stream) with the store resident in HBM and L2 flushed between steps; the
flush is outside the per-step events.  `e2e`: the same K steps through the
public API from a host store (pinned staging + one H2D copy per batch) with
the loss read back to the host every step, wall clock.  The reference arm
(`--impl reference`) times the FP64 CPU oracle on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

H, L, BATCH = 200, 6, 128
N_TRAIN, N_HELDOUT = 200_000, 20_000
SEED_DATA, SEED_TEACHER, SEED_STUDENT, SEED_ORDER = 10, 2, 3, 11
LR = 1e-3
METRIC = "train graphs/s"
WORKLOAD = "PNA GCNN training step: 200k synthetic molecular graphs (3-51 nodes, mean 18), 6 layers x 200, batch 128"
SM_COUNT, FP32_LANES_PER_SM = 152, 128
BM_ROWS, SM_CLOCK_HZ = 128, 2.07e9   # tensor-core GEMM tile rows; maximum SM clock


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dataset():
    gs = synth.molecules_lognormal(SEED_DATA, N_TRAIN + N_HELDOUT)
    return gs


def epoch_order(epoch: int = 0, replicate: int = 0) -> np.ndarray:
    seed = SEED_ORDER + 1000 * epoch + 100_000 * replicate
    return np.random.default_rng(seed).permutation(N_TRAIN).astype(np.int64)


def gemm_flops(n_nodes: int) -> float:
    """Algorithmic FLOPs of the step's dense GEMMs for a batch of n_nodes (all layers, fwd + bwd)."""
    per_layer = 2.0 * n_nodes * (H * 2 * H + 16 * H * H)          # forward: message, update
    per_layer += 2.0 * n_nodes * (16 * H * H + 3 * H * 5 * H + H * 2 * H + 3 * H * H)  # dW_U, dagg, dW_M, dx
    return L * per_layer


def agg_fwd_bytes(n_nodes: int, n_edges: int, precision: str = "fp32") -> float:
    """Compulsory bytes of one aggregation launch: P and Q rows read once, the CSR read, and the
    aggregates written (FP32 path: 5H FP32; BF16 path: the 15H scaled BF16 operand block)."""
    out = 15 * H * 2.0 if precision == "bf16" else 5 * H * 4.0
    return n_nodes * (2 * H * 4.0 + out) + (n_nodes + 1 + n_edges) * 4.0


def measured_hbm():
    """HBM copy bandwidth measured on the GB300s, else the documented fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback 6.8 TB/s"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={','.join(self.FIELDS)}",
                                          "--format=csv,noheader,nounits", "-lms", "200", "-i", str(gpu_index)],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"error": "nvidia-smi unavailable"}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"error": "no samples"}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle
def oracle_graphs_per_s(path: str, order: np.ndarray, budget_s: float):
    """Time the FP64 oracle's collation + fwd + bwd + Adam on a bounded sample of the workload:
    consecutive 128-graph batches of the epoch order until about budget_s seconds of host work."""
    import oracle
    cores = len(os.sched_getaffinity(0))
    ost = oracle.read_store(path)
    ost.y = synth.uniform_targets(SEED_DATA + 7, 0, len(ost.y), 1.0, 10.0)   # targets independent of the GPU
    d = oracle.Dims(H=H, L=L)
    p = synth.init_params(SEED_STUDENT, H, L).astype(np.float64)
    delta = oracle.delta_of(ost, order[:2048])

    def run(ids):
        t0 = time.perf_counter()
        b = oracle.collate(ost, ids, delta)
        loss, grad, _, _ = oracle.backward(d, p, b)
        th = p.copy()
        oracle.adam(th, grad, np.zeros_like(p), np.zeros_like(p), 1, lr=LR)
        return time.perf_counter() - t0

    batches = graphs = 0
    t = 0.0
    while t < budget_s and (batches + 1) * BATCH <= len(order):
        t += run(order[batches * BATCH:(batches + 1) * BATCH])
        graphs += BATCH
        batches += 1
    return {"value": graphs / t, "unit": "graphs/s", "cores": cores, "kind": "oracle",
            "sample": f"{batches} consecutive batches of {BATCH} graphs of the workload ({graphs} graphs), "
                      f"FP64 collation + fwd + bwd + AdamW each, {t:.1f} s, OpenMP over nodes on {cores} host cores"}


def oracle_single_thread(path: str, order: np.ndarray, budget_s: float):
    """The same oracle timing on one host thread: a child process with
    OMP_NUM_THREADS=1 (the OpenMP runtime reads it when the oracle loads)."""
    np.save(os.path.join(os.path.dirname(path), "order.npy"), order[:4096])
    code = ("import json, sys, numpy as np; sys.path.insert(0, %r); import bench; "
            "o = np.load(%r); print(json.dumps(bench.oracle_graphs_per_s(%r, o, %r)))"
            % (ROOT, os.path.join(os.path.dirname(path), "order.npy"), path, budget_s))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=budget_s * 4 + 120)
    if r.returncode != 0:
        return {"error": r.stderr[-300:]}
    out = json.loads(r.stdout.strip().splitlines()[-1])
    out["cores"] = 1
    out["sample"] = out["sample"].replace(f"on {len(os.sched_getaffinity(0))} host cores", "on 1 host thread")
    return out


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, bounded sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cores = len(os.sched_getaffinity(0))
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    import oracle
    gs = dataset()
    tmp = tempfile.mkdtemp(prefix="gcnn_ref_")
    path = os.path.join(tmp, "train.gcnn")
    synth.write_store(path, gs)
    ost = oracle.read_store(path)
    ost.y = synth.uniform_targets(SEED_DATA + 7, 0, len(ost.y), 1.0, 10.0)
    order = epoch_order(0)
    d = oracle.Dims(H=H, L=L)
    p = synth.init_params(SEED_STUDENT, H, L).astype(np.float64)
    m, v = np.zeros_like(p), np.zeros_like(p)
    delta = oracle.delta_of(ost, order[:2048])

    def step(ids, t):
        b = oracle.collate(ost, ids, delta)
        loss, grad, _, _ = oracle.backward(d, p, b)
        oracle.adam(p, grad, m, v, t, lr=LR)

    t0 = time.perf_counter()
    step(order[:2], 1)
    per_graph = (time.perf_counter() - t0) / 2
    budget = args.ref_seconds
    gps = int(max(1, min(BATCH, budget / max(per_graph * (args.steps + args.warmup), 1e-9))))
    pos = 2
    for w in range(args.warmup):
        step(order[pos:pos + gps], 2 + w)
        pos += gps
    t0 = time.perf_counter()
    for k in range(args.steps):
        step(order[pos:pos + gps], 2 + args.warmup + k)
        pos = (pos + gps) % (N_TRAIN - BATCH)
    dt = time.perf_counter() - t0
    value = args.steps * gps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "graphs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "graphs_per_step": gps, "hidden": H, "layers": L},
            "cpu_baseline": {"value": value, "unit": "graphs/s", "cores": cores, "kind": "oracle",
                             "sample": f"{gps} graphs per step (bounded sample of the 128-graph batch)"},
            "e2e": {"value": value, "unit": "graphs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
def make_targets(g, st, delta, n_graphs, gpu_batch=2048):
    """Teacher (same architecture, seed 2) predictions over every graph, mapped to [1, 10]."""
    import torch
    ids_all = np.arange(n_graphs, dtype=np.int64)
    caps = [st.batch_size(ids_all[i:i + gpu_batch]) for i in range(0, n_graphs, gpu_batch)]
    Nc = max(c[0] for c in caps)
    Ec = max(c[1] for c in caps)
    t = g.Context(g.make_config(H, L, gpu_batch, Nc, Ec, delta=delta))
    t.set_params(synth.init_params(SEED_TEACHER, H, L))
    out = torch.empty(n_graphs, device="cuda")
    for i in range(0, n_graphs, gpu_batch):
        b = t.collate(st, ids_all[i:i + gpu_batch])
        t.forward(b, out[i:i + b.n_graphs], train=False)
    y = out.cpu().numpy().astype(np.float64)
    t.close()
    lo, hi = y.min(), y.max()
    return (1.0 + 9.0 * (y - lo) / max(hi - lo, 1e-30)).astype(np.float32)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


class Workload:
    """The 200k-graph store (device-resident), its teacher targets, the epoch order, capacities.

    One process: the seeded epoch order in batches of 128.  Data parallel (ddp):
    the package's ShardedSampler over the same graphs, 128 per process and step,
    and capacities that cover every process's share."""

    def __init__(self, g, rank: int, world: int = 1, ddp: bool = False):
        gs = dataset()
        self.counts = np.diff(gs.node_ptr)[:N_TRAIN]
        self.tmp = tempfile.mkdtemp(prefix="gcnn_bench_")
        self.path = os.path.join(self.tmp, "train.gcnn")
        synth.write_store(self.path, gs)
        self.st = g.Store(self.path)
        self.st.to_device()
        self.delta = self.st.delta(np.arange(N_TRAIN))
        self.y = make_targets(g, self.st, self.delta, N_TRAIN + N_HELDOUT)
        self.st.set_targets(self.y)
        self.sampler = None
        if ddp:
            from paper_2207_11333_gb300.ddp import ShardedSampler
            self.sampler = ShardedSampler(N_TRAIN, BATCH, world, rank, SEED_ORDER, node_counts=self.counts)
            shards = [self.sampler.shard(k).ids for k in range(len(self.sampler))]
            self.order = np.concatenate(shards)
            sizes = [self.st.batch_size(ids) for ids in shards]
        else:
            self.order = np.ascontiguousarray(epoch_order(0))
        self.n_train = len(self.order)
        self.nb = (self.n_train + BATCH - 1) // BATCH
        if not ddp:
            sizes = [self.st.batch_size(self.order[i * BATCH:(i + 1) * BATCH]) for i in range(self.nb)]
        self.Nc = (max(s[0] for s in sizes) + 255) // 256 * 256
        self.Ec = (max(s[1] for s in sizes) + 511) // 512 * 512


def make_ctx(g, wl: Workload, precision: str, flags: int = 0):
    prec = g.PREC_BF16 if precision == "bf16" else g.PREC_FP32
    ctx = g.Context(g.make_config(H, L, BATCH, wl.Nc, wl.Ec, delta=wl.delta, precision=prec, flags=flags))
    ctx.set_params(synth.init_params(SEED_STUDENT, H, L))
    ctx.set_order(wl.st, wl.order)
    return ctx


def batch_at(ctx, wl: Workload, k: int):
    i = k % wl.nb
    return ctx.collate_range(wl.st, i * BATCH, min(BATCH, wl.n_train - i * BATCH))


def train_at(ctx, wl: Workload, k: int, loss_acc):
    """Training step k: collation of batch k of the epoch order and the step in one graph launch."""
    i = k % wl.nb
    return ctx.train_step_range(wl.st, i * BATCH, min(BATCH, wl.n_train - i * BATCH), LR, loss_acc)


def timed_steps(ctx, wl, steps, warmup, flush, loss_acc, dist=None, gpu_index=None):
    """Device time of `steps` training steps (per-step CUDA events, L2 flushed between steps)."""
    import torch
    for k in range(warmup):
        train_at(ctx, wl, k, loss_acc)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_index) if gpu_index is not None else None
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    graphs = 0
    torch.cuda.nvtx.range_push("timed")
    t_wall = time.perf_counter()
    for k in range(steps):
        flush.zero_()
        evs[k][0].record()
        b = train_at(ctx, wl, warmup + k, loss_acc)
        evs[k][1].record()
        graphs += b.n_graphs
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    torch.cuda.nvtx.range_pop()
    clocks = sampler.stop() if sampler else None
    dev_s = sum(a.elapsed_time(b) for a, b in evs) / 1e3
    if dist:
        tmax = torch.tensor([dev_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        gsum = torch.tensor([float(graphs)], dtype=torch.float64, device="cuda")
        dist.all_reduce(gsum, op=dist.ReduceOp.SUM)
        dev_s, total = float(tmax.item()), float(gsum.item())
    else:
        total = float(graphs)
    # the collation's two kernels are part of the step's graph
    return {"value": total / dev_s, "dev_s": dev_s, "graphs": total, "wall_s": wall, "clocks": clocks,
            "kernels_per_step": ctx.step_kernel_count()}


def timed_ddp_steps(g, ctx, wl, steps, warmup, flush, loss_acc, dist, gpu_index, store=None, e2e=False):
    """Data-parallel steps (Sec. 4, Fig. 4) through the package's DataParallelTrainer:
    per process its share of every global batch, collated from the store, the
    loss gradient scaled by that share, the backward, each gradient bucket
    all-reduced over NCCL as soon as it is final, then AdamW.  Device time per
    step from CUDA events (L2 flushed between steps, outside the events), the
    maximum over processes; with e2e, wall clock of the steps from a host store
    with every step's loss read back to the host."""
    import torch
    from paper_2207_11333_gb300.ddp import DataParallelTrainer
    tr = DataParallelTrainer(ctx, store or wl.st, wl.sampler)
    n_steps = len(wl.sampler)
    for k in range(warmup):
        tr.step(k % n_steps, LR, loss_acc)
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_index) if (gpu_index is not None and not e2e) else None
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    pinned = torch.zeros(3, dtype=torch.float64).pin_memory()
    graphs = h2d = 0
    mine = []
    t_wall = time.perf_counter()
    for k in range(steps):
        if not e2e:
            flush.zero_()
        evs[k][0].record()
        sh = tr.step((warmup + k) % n_steps, LR, loss_acc)
        evs[k][1].record()
        if e2e:
            pinned.copy_(loss_acc, non_blocking=True)
            torch.cuda.current_stream().synchronize()
            assert math.isfinite(float(pinned[0]))
            mine.append(sh.ids)
        graphs += sum(sh.graphs)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    for ids in mine:        # bytes staged and copied per step: offsets, targets, types, local edges
        n_atoms, n_edges = wl.st.batch_size(ids)
        h2d += 16 * (len(ids) + 1) + 4 * len(ids) + n_atoms + 2 * n_edges
    clocks = sampler.stop() if sampler else None
    dev_s = sum(a.elapsed_time(b) for a, b in evs) / 1e3
    t = torch.tensor([dev_s, wall], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dev_s, wall = float(t[0]), float(t[1])
    out = {"value": graphs / (wall if e2e else dev_s), "dev_s": dev_s, "graphs": float(graphs), "wall_s": wall,
           "clocks": clocks, "h2d_bytes_per_step": h2d / steps}
    # kernels per step from the library's kernel timeline over one more step
    ctx.timeline_enable(4096)
    ctx.timeline_read()
    tr.step(0, LR, loss_acc)
    torch.cuda.synchronize()
    ids, _ = ctx.timeline_read()
    ctx.timeline_enable(0)
    out["kernels_per_step"] = len(ids)
    return out


def gemm_traffic():
    """DRAM bytes per GEMM launch from the committed ncu record
    (profiles/tma_gemm_bf16_train_step_200k.json), or None when the GEMM
    kernel's source has changed since those counters were taken."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "tma_gemm_bf16_train_step_200k.json")) as f:
            rec = json.load(f)
        with open(os.path.join(ROOT, rec["source"]), "rb") as f:
            src = hashlib.sha256(f.read()).hexdigest()
    except (OSError, ValueError, KeyError):
        return None
    return float(rec["dram_bytes_per_launch"]) if rec.get("source_sha256") == src else None


def kernel_profile(g, wl, n_steps, warmup, flush, loss_acc, precision):
    """Per-kernel durations inside the captured step, from the library's kernel timeline.

    Every library kernel records the device clock once its dependency on the
    previous kernel is satisfied (the previous kernel's completion), so in a
    serial graph the difference of consecutive records is a kernel's duration
    as it runs in the step.  The timed step overlaps the BF16 weight-gradient
    work on a second stream; these durations come from the same step on one
    stream (GCNN_FLAG_SERIAL, same kernels and launch shapes).  The library
    appends a one-thread marker kernel after the step while the timeline is
    on, so the optimiser (the step's last kernel) is timed too, with the
    graph's completion latency included; the collation kernels are the
    graph's first launches (gcnn_train_step_range).  Phases
    follow the launch order: collation, forward (embedding through the head
    and loss), backward (head gradient through the embedding gradient) and
    the optimiser."""
    import torch
    from collections import Counter, defaultdict
    ctx = make_ctx(g, wl, precision, g.FLAG_SERIAL)
    for k in range(warmup):
        train_at(ctx, wl, k, loss_acc)
    torch.cuda.synchronize()
    ctx.timeline_enable(256 * n_steps)
    ctx.timeline_read()
    flops = agg_bytes = 0.0
    dur, cnt, ph = defaultdict(float), Counter(), defaultdict(float)
    for k in range(n_steps):
        flush.zero_()
        b = train_at(ctx, wl, warmup + k, loss_acc)
        torch.cuda.synchronize()
        ids, t = ctx.timeline_read()
        phase = "collate"
        for i in range(len(ids) - 1):
            name = g.KERNELS.get(int(ids[i]), str(int(ids[i])))
            phase = {"embed": "forward", "head_grad": "backward", "adam": "optimizer"}.get(name, phase)
            dur[name] += (t[i + 1] - t[i]) * 1e-9
            cnt[name] += 1
            ph[phase] += (t[i + 1] - t[i]) * 1e-9
        flops += gemm_flops(b.n_nodes)
        agg_bytes += L * agg_fwd_bytes(b.n_nodes, b.n_edges, precision)
    ctx.timeline_enable(0)
    ctx.check()
    ctx.close()
    out = {"kernel_ms_per_step": {k: {"ms": 1e3 * v / n_steps, "launches": cnt[k] // n_steps}
                                  for k, v in sorted(dur.items(), key=lambda x: -x[1])},
           "phase_us_per_step": {k: round(1e6 * v / n_steps, 1) for k, v in ph.items()},
           "kernel_timing": "library kernel timeline (device clock at each kernel's start after its dependency "
                            "wait) over the step on one stream; L2 flushed before each step"}
    peaks = measured_peaks()
    if precision == "bf16":
        gemm_s = sum(v for k, v in dur.items() if k.startswith("gemm_tc"))
        launches = sum(c for k, c in cnt.items() if k.startswith("gemm_tc_") and k != "gemm_tc_reduce") / n_steps
        achieved = flops / gemm_s / 1e12
        peak = float(peaks.get("bf16_tflops", 1900.0))
        src = "measured (MEASURED_PEAKS.json bf16_tflops, burst)" if "bf16_tflops" in peaks else "fallback 1.9 PFLOP/s"
        out["roofline"] = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                           "frac": achieved / peak, "traffic": gemm_traffic(), "traffic_unit": "DRAM bytes per launch",
                           "peak_source": src, "launches_per_step": launches,
                           "kernel": "tma_gemm_kernel<epilogue, cluster> (all dense GEMMs of the step, BF16 tcgen05, "
                                     "FP32 accumulate, split-K summed in thread-block clusters)"}
    else:
        gemm_s = sum(v for k, v in dur.items() if k.startswith("gemm_simt"))
        achieved = flops / gemm_s / 1e12
        derived = SM_COUNT * FP32_LANES_PER_SM * 2 * 2070.0 * 1e6 / 1e12
        peak = g.ffma_peak(8192)
        out["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                           "frac": achieved / peak, "traffic": None,
                           "peak_source": "measured live: gcnn_ffma_peak (independent FFMA chains on every SM); "
                                          f"derived 152 SMs x 128 lanes x 2 FLOP x 2070 MHz = {derived:.1f}",
                           "kernel": "sgemm_kernel + splitk_reduce (all dense GEMMs of the step, FP32 FFMA)"}
    hbm, hbm_src = measured_hbm()
    a_gbs = agg_bytes / dur["agg_fwd"] / 1e9
    out["roofline_aggregate"] = {"bound": "hbm", "achieved": a_gbs, "peak": hbm, "unit": "GB/s", "frac": a_gbs / hbm,
                                 "traffic": None, "peak_source": hbm_src, "kernel": "aggregate_fwd_kernel",
                                 "note": "128-graph batches fit in L2; the HBM figure needs a >L2 batch"}
    return out


def e2e_steps(g, ctx, wl, steps, loss_acc):
    """The same steps through the public API from a host store: pinned staging + H2D per batch,
    and every step's loss read back to pinned host memory.  The host reads step k's loss once
    step k + 1 is queued (a two-deep ring of pinned buffers and events), so its staging of
    the next batch overlaps the device's step, as in a training loop that logs every loss."""
    import torch
    sh = g.Store(wl.path)          # host-resident twin
    sh.set_targets(wl.y)
    pinned = [torch.zeros(3, dtype=torch.float64).pin_memory() for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]
    for k in range(3):
        ctx.train_step(ctx.collate(sh, wl.order[k * BATCH:(k + 1) * BATCH]), LR, loss_acc)
    torch.cuda.synchronize()
    h2d = 0
    n = 0
    losses = []
    t0 = time.perf_counter()
    for k in range(steps):
        i = k % wl.nb
        b = ctx.collate(sh, wl.order[i * BATCH:(i + 1) * BATCH])
        ctx.train_step(b, LR, loss_acc)
        pinned[k % 2].copy_(loss_acc, non_blocking=True)
        done[k % 2].record()
        if k > 0:
            done[(k - 1) % 2].synchronize()
            losses.append(float(pinned[(k - 1) % 2][0]))
        n += b.n_graphs
        h2d += 16 * (b.n_graphs + 1) + 4 * b.n_graphs + b.n_nodes + 2 * b.n_edges
    done[(steps - 1) % 2].synchronize()
    losses.append(float(pinned[(steps - 1) % 2][0]))
    dt = time.perf_counter() - t0
    assert len(losses) == steps and all(math.isfinite(v) for v in losses)
    return {"value": n / dt, "unit": "graphs/s", "h2d_bytes_per_step": h2d / steps, "d2h_bytes_per_step": 24,
            "steps": steps, "path": "gcnn_collate from a host store (pinned staging, one H2D) + gcnn_train_step "
                                    "+ every step's loss copied to pinned host memory and read one step later"}


# ------------------------------------------------------------------ large batches
def aggregate_large(g, reps: int = 5, G: int = 60_000):
    """HBM throughput of the aggregation kernels on a batch far larger than L2.

    60,000 molecules (about 1.1M atoms, 2.4M directed edges) collated on the device,
    random P|Q rows at H = 200.  Compulsory bytes: the forward reads P and Q and
    writes 5H aggregates per node; the backward reads P|Q, the four stored
    statistics and the 5H incoming gradient and writes dP|dQ (13H floats per node)
    plus the CSR indices.  "backward" is the whole-graph entry point (fused over
    chunks of graphs, per-edge gradients in shared memory); "backward_pair" is the
    edge + gather pair, whose per-edge buffer (written and read back, 2 E H floats)
    is counted on top for it.
    """
    import torch
    gs = synth.molecules_lognormal(SEED_DATA + 100, G)
    tmp = tempfile.mkdtemp(prefix="gcnn_large_")
    path = os.path.join(tmp, "large.gcnn")
    synth.write_store(path, gs)
    st = g.Store(path)
    N, E = gs.n_nodes, gs.n_edges
    c = g.Context(g.make_config(8, 1, G, N, E, delta=st.delta()))
    b = c.collate(st, np.arange(G))
    rp, col, rev, no = b.tensor("row_ptr"), b.tensor("col"), b.tensor("rev"), b.tensor("node_off")
    Hl = H
    gen = torch.Generator(device="cuda").manual_seed(5)
    PQ = torch.randn(N, 2 * Hl, device="cuda", generator=gen)
    agg = g.aggregate_fwd(PQ, rp, col)
    dagg = torch.randn(N, 5 * Hl, device="cuda", generator=gen)
    dPQ = g.aggregate_bwd(PQ, agg, dagg, rp, col, rev, node_off=no)
    same = bool(torch.equal(dPQ, g.aggregate_bwd(PQ, agg, dagg, rp, col, rev)))
    torch.cuda.synchronize()
    fwd_bytes = N * (2 * Hl + 5 * Hl) * 4.0 + (N + 1 + E) * 4.0
    bwd_bytes = N * (2 * Hl + 4 * Hl + 5 * Hl + 2 * Hl) * 4.0 + (N + 1 + 2 * E + G + 1) * 4.0
    pair_bytes = bwd_bytes + 2.0 * E * Hl * 4
    out = {}
    for name, fn, nbytes in (("forward", lambda: g.aggregate_fwd(PQ, rp, col), fwd_bytes),
                             ("backward", lambda: g.aggregate_bwd(PQ, agg, dagg, rp, col, rev, node_off=no),
                              bwd_bytes),
                             ("backward_pair", lambda: g.aggregate_bwd(PQ, agg, dagg, rp, col, rev), pair_bytes)):
        fn()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        t = min(ts)
        out[name] = {"ms": 1e3 * t, "algorithmic_bytes": nbytes, "GB_s": nbytes / t / 1e9}
    hbm, src = measured_hbm()
    for v in out.values():
        v["frac_of_hbm"] = v["GB_s"] / hbm
    out.update({"nodes": N, "edges": E, "hidden": Hl, "peak_GB_s": hbm, "peak_source": src,
                "backward_equals_pair_bitwise": same,
                "note": "gcnn_op_aggregate_fwd / _bwd_graphs / _bwd through the C ABI; best of the timed launches, "
                        "CUDA events; the scratch of the backward is allocated inside the timed call"})
    del PQ, agg, dagg, dPQ
    c.close()
    return out


def loading_study(g, n_graphs: int = 20_000, batches: int = 60):
    """Data loading (Sec. 4, Fig. 5 bottom): one file per molecule against the packed
    store of global arrays.  n_graphs molecules of the workload's size distribution are
    written one file each, packed by gcnn_store_pack with 1 and with all host threads,
    and `batches` random 128-graph batches are collated three ways, each followed by a
    device synchronisation: from the files (gcnn_collate_files: one open + read per
    molecule), from the packed store in pinned host memory (one copy per batch) and from
    the device-resident store.  The files were just written, so they are read from the
    page cache: the per-file figure is the file-system call overhead, not disk time."""
    import shutil
    import torch
    gs = synth.molecules_lognormal(SEED_DATA + 300, n_graphs)
    gs.y = synth.uniform_targets(SEED_DATA + 301, 0, n_graphs, 1.0, 10.0)
    tmp = tempfile.mkdtemp(prefix="gcnn_files_")
    out = {"graphs": n_graphs, "batch": BATCH, "batches": batches}
    try:
        t0 = time.perf_counter()
        paths = synth.write_graph_files(os.path.join(tmp, "files"), gs)
        out["write_files_s"] = time.perf_counter() - t0
        cores = len(os.sched_getaffinity(0))
        packed = os.path.join(tmp, "packed.gcnn")
        for threads in sorted({1, cores}):
            t0 = time.perf_counter()
            g.store_pack(paths, packed, threads)
            out[f"pack_s_{threads}_threads"] = time.perf_counter() - t0
        t0 = time.perf_counter()
        st = g.Store(packed)
        out["open_packed_s"] = time.perf_counter() - t0
        rng = np.random.default_rng(7)
        sets = [rng.integers(0, n_graphs, BATCH) for _ in range(batches)]
        sizes = [st.batch_size(ids) for ids in sets]
        Nc = (max(sz[0] for sz in sizes) + 255) // 256 * 256
        Ec = (max(sz[1] for sz in sizes) + 511) // 512 * 512
        ctx = g.Context(g.make_config(H, L, BATCH, Nc, Ec, delta=st.delta()))
        ways = (("per_graph_files", lambda ids: ctx.collate_files([paths[i] for i in ids])),
                ("packed_store_host", lambda ids: ctx.collate(st, ids)))
        for name, fn in ways + (("packed_store_device", None),):
            if name == "packed_store_device":
                st.to_device()
                fn = lambda ids: ctx.collate(st, ids)  # noqa: E731
            fn(sets[0])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for ids in sets:
                fn(ids)
                torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            out[name] = {"ms_per_batch": 1e3 * dt / batches, "graphs_per_s": batches * BATCH / dt}
        ctx.check()
        ctx.close()
        out["files_over_packed_host"] = out["per_graph_files"]["ms_per_batch"] / out["packed_store_host"]["ms_per_batch"]
        out["note"] = "wall time per collated batch incl. device sync; files read from the page cache"
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
    return out


def variants_study(g, wl: Workload, flush, precision: str, steps: int = 200, warmup: int = 10):
    """The next rows of the path on the same workload and step: bond features (F = 4 per
    edge in the message, Sec. 3.1 / Table 1 edge attributes) and the node-level head
    (Sec. 3.1 node-level properties), alone and together; train graphs/s from the same
    per-step CUDA events as the headline value."""
    import torch
    from types import SimpleNamespace
    gs = dataset()
    gs.y = wl.y
    gs.ynode = synth.uniform(SEED_DATA + 401, 0, gs.n_nodes, -1.0, 1.0).astype(np.float32)
    stores = {}
    for F in (0, 4):  # node targets, without and with bond features
        gs.eattr = synth.bond_features(SEED_DATA + 400, gs, 4, -1.0, 1.0) if F else None
        path = os.path.join(wl.tmp, f"variants_{F}.gcnn")
        synth.write_store(path, gs)
        stores[F] = g.Store(path)
        stores[F].to_device()
    prec = g.PREC_BF16 if precision == "bf16" else g.PREC_FP32
    out = {"precision": precision, "steps": steps}
    for name, F, nh in (("bond_features_4", 4, 0), ("node_head", 0, 1), ("both", 4, 1)):
        st = stores[F]
        vw = SimpleNamespace(st=st, nb=wl.nb, n_train=wl.n_train)
        ctx = g.Context(g.make_config(H, L, BATCH, wl.Nc, wl.Ec, delta=wl.delta, precision=prec, edge_features=F,
                                      node_head=nh))
        p = synth.init_params(SEED_STUDENT, H, L, F=F)
        if nh:  # node head block: from a multiple of 4 floats, drawn like a graph head
            p = np.concatenate([p, np.zeros((p.size + 3) // 4 * 4 - p.size, np.float32),
                                synth.init_params(SEED_STUDENT + 1, H, 1)[-(H * H + 2 * H + 1):]])
        ctx.set_params(p)
        ctx.set_order(st, wl.order)
        acc = torch.zeros(5, dtype=torch.float64, device="cuda")
        r = timed_steps(ctx, vw, steps, warmup, flush, acc)
        ctx.check()
        ctx.close()
        out[name] = {"graphs_per_s": r["value"], "ms_per_step": 1e3 * r["dev_s"] / steps}
    for st in stores.values():
        st.close()
    return out


def recompute_study(g, precision: str, steps: int = 20):
    """Per-layer recompute at H = 256, L = 6, 1024 graphs of 3-51 atoms per batch:
    step time and device memory with and without it."""
    import torch
    Hr, Lr, Br = 256, 6, 1024
    gs = synth.molecules_lognormal(SEED_DATA + 200, 16 * Br)
    tmp = tempfile.mkdtemp(prefix="gcnn_recompute_")
    path = os.path.join(tmp, "rc.gcnn")
    synth.write_store(path, gs)
    st = g.Store(path)
    st.to_device()
    delta = st.delta()
    sizes = [st.batch_size(np.arange(i * Br, (i + 1) * Br)) for i in range(16)]
    Nc = max(s[0] for s in sizes) + 256
    Ec = max(s[1] for s in sizes) + 512
    prec = g.PREC_BF16 if precision == "bf16" else g.PREC_FP32
    out = {"hidden": Hr, "layers": Lr, "batch_graphs": Br, "precision": precision,
           "mean_nodes_per_batch": float(np.mean([s[0] for s in sizes]))}
    params = synth.init_params(SEED_STUDENT, Hr, Lr)
    for rc in (0, 1):
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        c = g.Context(g.make_config(Hr, Lr, Br, Nc, Ec, delta=delta, precision=prec, recompute=rc))
        free1 = torch.cuda.mem_get_info()[0]
        c.set_params(params)
        c.set_order(st, np.arange(16 * Br))
        for k in range(3):
            c.train_step(c.collate_range(st, (k % 16) * Br, Br), LR)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for k in range(steps):
            c.train_step(c.collate_range(st, (k % 16) * Br, Br), LR)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out["recompute" if rc else "stored"] = {"ms_per_step": ms, "graphs_per_s": Br / (ms / 1e3),
                                                "arena_bytes": c.memory_bytes(), "device_bytes_taken": free0 - free1}
        c.close()
    return out


# ------------------------------------------------------------------ precision study
def precision_study(g, epochs: int, lr: float, seeds: int = 1):
    """FP32 and BF16 paths trained from the same initial parameters on the same epoch
    orders of the 200k-graph set, the learning rate decayed over the run by a half
    cosine from `lr` to zero (so that the last epochs settle instead of moving with
    the step size); training MSE per epoch and MAE on the held-out 20k.  With
    seeds > 1 the pair is trained again from other initial parameters and epoch
    orders, and the comparison figure is the relative difference of the two
    paths' final held-out MAE, averaged over the seeds, with its standard error."""
    import torch
    wl = Workload(g, 0, 1)
    held = np.arange(N_TRAIN, N_TRAIN + N_HELDOUT, dtype=np.int64)
    hs = [wl.st.batch_size(held[i:i + BATCH]) for i in range(0, N_HELDOUT, BATCH)]
    Nc = max(wl.Nc, (max(s[0] for s in hs) + 255) // 256 * 256)
    Ec = max(wl.Ec, (max(s[1] for s in hs) + 511) // 512 * 512)
    y_held = wl.y[held].astype(np.float64)
    out = {"epochs": epochs, "train_graphs": N_TRAIN, "heldout_graphs": N_HELDOUT, "batch": BATCH, "lr": lr,
           "lr_schedule": "half cosine from lr to 0 over all steps", "seeds": seeds}
    steps_per_epoch = (N_TRAIN + BATCH - 1) // BATCH
    total = epochs * steps_per_epoch

    def train(prec, r):
        c = g.Context(g.make_config(H, L, BATCH, Nc, Ec, delta=wl.delta,
                                    precision=g.PREC_BF16 if prec == "bf16" else g.PREC_FP32))
        c.set_params(synth.init_params(SEED_STUDENT + 100 * r, H, L))
        pred = torch.empty(N_HELDOUT, device="cuda")
        hist = []
        t0 = time.perf_counter()
        for ep in range(epochs):
            order = epoch_order(ep, r)
            c.set_order(wl.st, order)
            acc = torch.zeros(3, dtype=torch.float64, device="cuda")
            for j, i in enumerate(range(0, N_TRAIN, BATCH)):
                lr_k = 0.5 * lr * (1.0 + math.cos(math.pi * (ep * steps_per_epoch + j) / total))
                c.train_step(c.collate_range(wl.st, i, min(BATCH, N_TRAIN - i)), lr_k, acc)
            a = acc.cpu().numpy()
            for i in range(0, N_HELDOUT, BATCH):
                b = c.collate(wl.st, held[i:i + BATCH])
                c.forward(b, pred[i:i + b.n_graphs], train=False)
            err = pred.cpu().numpy().astype(np.float64) - y_held
            hist.append({"epoch": ep + 1, "train_mse": a[0] / a[2], "train_mae": a[1] / a[2],
                         "heldout_mae": float(np.mean(np.abs(err))), "heldout_rmse": float(np.sqrt(np.mean(err ** 2)))})
            log(f"[precision] seed {r} {prec} epoch {ep + 1}: {hist[-1]}")
        c.check()
        c.close()
        return {"history": hist, "seconds": time.perf_counter() - t0}

    reps = []
    for r in range(seeds):
        run = {p: train(p, r) for p in ("fp32", "bf16")}
        if r == 0:
            out.update(run)
        f32, f16 = run["fp32"]["history"][-1]["heldout_mae"], run["bf16"]["history"][-1]["heldout_mae"]
        reps.append({"seed": r, "fp32_heldout_mae": f32, "bf16_heldout_mae": f16, "rel_diff": (f16 - f32) / f32})
    h32, h16 = out["fp32"]["history"], out["bf16"]["history"]
    out["final_train_mse_rel_diff"] = (h16[-1]["train_mse"] - h32[-1]["train_mse"]) / h32[-1]["train_mse"]
    out["final_heldout_mae_rel_diff"] = (h16[-1]["heldout_mae"] - h32[-1]["heldout_mae"]) / h32[-1]["heldout_mae"]
    b32, b16 = min(h["heldout_mae"] for h in h32), min(h["heldout_mae"] for h in h16)
    out["best_heldout_mae_rel_diff"] = (b16 - b32) / b32
    m32, m16 = (float(np.mean([h["heldout_mae"] for h in hh[-3:]])) for hh in (h32, h16))
    out["last3_heldout_mae"] = {"fp32": m32, "bf16": m16, "rel_diff": (m16 - m32) / m32}
    d = np.array([x["rel_diff"] for x in reps])
    out["replicates"] = reps
    out["final_heldout_mae_rel_diff_over_seeds"] = {
        "mean": float(d.mean()), "std_err": float(d.std(ddof=1) / np.sqrt(len(d))) if len(d) > 1 else None,
        "fp32_mean": float(np.mean([x["fp32_heldout_mae"] for x in reps])),
        "bf16_mean": float(np.mean([x["bf16_heldout_mae"] for x in reps]))}
    return out


# ------------------------------------------------------------------ serving
SERVE_POOL, SEED_SERVE = 100_000, 30


def arrival_schedule(lam: float, seconds: float, n_pool: int, seed: int):
    """Poisson arrivals at rate lam for `seconds`; request sizes log-uniform in 1..4096 molecules."""
    rng = np.random.default_rng(seed)
    n = max(1, int(lam * seconds))
    t = np.cumsum(rng.exponential(1.0 / lam, n))
    size = np.clip(np.floor(np.exp(rng.uniform(0.0, np.log(4097.0), n))), 1, 4096).astype(np.int64)
    start = rng.integers(0, n_pool - 4096, n)
    keep = t <= seconds
    return t[keep], size[keep], start[keep]


def summarize(lat_us, molecules, elapsed, offered, refused, lam):
    lat = np.sort(np.asarray(lat_us, np.float64)) / 1e3
    pct = (lambda q: float(lat[min(len(lat) - 1, int(q * len(lat)))]) if len(lat) else None)
    return {"lambda_req_s": lam, "requests_done": len(lat), "requests_offered": offered, "refused": refused,
            "served_graphs_per_s": molecules / elapsed if elapsed > 0 else 0.0, "p50_ms": pct(0.50),
            "p99_ms": pct(0.99), "elapsed_s": elapsed}


def serve_rates(g, model_ctx, pool, rates, seconds, precision, slots=4):
    """Continuous-batching server under Poisson load."""
    prec = g.PREC_BF16 if precision == "bf16" else g.PREC_FP32
    srv = g.Server(model_ctx, n_slots=slots, buckets=(1024, 4096, 16384, 65536), max_graphs=4096, precision=prec,
                   queue_nodes=1 << 22)
    warm = srv.submit(*g.request_arrays(pool, 0, 4096))   # every bucket's graph is captured at creation
    srv.wait(warm)
    for b in (1, 60, 300):
        srv.wait(srv.submit(*g.request_arrays(pool, 0, b)))
    out = []
    for r_i, lam in enumerate(rates):
        tm0 = srv.timing()
        t_arr, size, start = arrival_schedule(lam, seconds, pool.n_graphs, SEED_SERVE + r_i)
        pending, lat, mols, refused = [], [], 0, 0
        i = 0
        t0 = time.perf_counter()
        while i < len(t_arr) or pending:
            now = time.perf_counter() - t0
            while i < len(t_arr) and t_arr[i] <= now:
                t = srv.submit(*g.request_arrays(pool, int(start[i]), int(size[i])))
                if t is None:
                    refused += 1
                else:
                    pending.append((t, int(size[i])))
                i += 1
            still = []
            for t, n in pending:
                r = srv.poll(t)
                if r is None:
                    still.append((t, n))
                else:
                    lat.append(r[1])
                    mols += n
            pending = still
            if now > seconds + max(5.0, seconds):   # bounded drain
                break
            if not still and i < len(t_arr):
                time.sleep(max(0.0, min(0.001, t_arr[i] - (time.perf_counter() - t0))))
        elapsed = time.perf_counter() - t0
        res = summarize(lat, mols, elapsed, len(t_arr), refused, lam)
        tm1 = srv.timing()
        nb = max(1, tm1["batches"] - tm0["batches"])
        res["batches"] = tm1["batches"] - tm0["batches"]
        res["atoms_per_batch"] = (tm1["atoms"] - tm0["atoms"]) / nb
        res["scheduler_us_per_batch"] = (tm1["host_us"] - tm0["host_us"]) / nb
        res["device_us_per_batch"] = (tm1["device_us"] - tm0["device_us"]) / nb
        # fraction of the wall time the scheduler thread spent forming and
        # launching batches, and the mean number of batches on the device
        res["scheduler_busy"] = (tm1["host_us"] - tm0["host_us"]) / (1e6 * elapsed)
        res["device_batches_in_flight"] = (tm1["device_us"] - tm0["device_us"]) / (1e6 * elapsed)
        out.append(res)
    stats = srv.stats()
    srv.close()
    return out, stats


def baseline_rates(g, params, delta, pool_path, pool, rates, seconds):
    """Plain FP32 path, one request per launch in arrival order (collate from host + forward + read back)."""
    import torch
    n_max = 4096 * 80
    ctx = g.Context(g.make_config(H, L, 4096, n_max, 4 * n_max + 1024, delta=delta))
    ctx.set_params(params)
    st = g.Store(pool_path)
    pred = torch.empty(4096, device="cuda")
    host = torch.empty(4096, dtype=torch.float32).pin_memory()
    out = []
    for r_i, lam in enumerate(rates):
        t_arr, size, start = arrival_schedule(lam, seconds, pool.n_graphs, SEED_SERVE + r_i)
        lat, mols = [], 0
        t0 = time.perf_counter()
        for i in range(len(t_arr)):
            now = time.perf_counter() - t0
            if now < t_arr[i]:
                time.sleep(t_arr[i] - now)
            if time.perf_counter() - t0 > seconds + max(5.0, seconds):   # bounded drain
                break
            n = int(size[i])
            b = ctx.collate(st, np.arange(start[i], start[i] + n))
            ctx.forward(b, pred, train=False)
            host[:n].copy_(pred[:n], non_blocking=True)
            torch.cuda.current_stream().synchronize()
            lat.append(1e6 * (time.perf_counter() - t0 - t_arr[i]))
            mols += n
        elapsed = time.perf_counter() - t0
        out.append(summarize(lat, mols, elapsed, len(t_arr), 0, lam))
    ctx.close()
    return out


def run_serving(g, model_ctx, delta, params, args):
    pool = synth.molecules_uniform(SEED_SERVE, SERVE_POOL, 5, 80)
    tmp = tempfile.mkdtemp(prefix="gcnn_serve_")
    path = os.path.join(tmp, "pool.gcnn")
    synth.write_store(path, pool)
    rates = [float(x) for x in args.serve_rates.split(",")]
    res, stats = serve_rates(g, model_ctx, pool, rates, args.serve_seconds, args.precision, args.serve_slots)
    base_s = min(args.serve_seconds, args.baseline_seconds)
    base = baseline_rates(g, params, delta, path, pool, rates, base_s)
    return {"workload": "Poisson arrivals; 1-4096 molecules per request (log-uniform), 5-80 atoms each; "
                        f"{args.serve_seconds:g} s per rate (baseline {base_s:g} s per rate)",
            "server": {"precision": args.precision, "slots": args.serve_slots, "buckets_nodes": [1024, 4096, 16384, 65536],
                       "rates": res, "totals": stats},
            "baseline_fp32_one_request_per_launch": {"rates": base}}


def gemm_study(args):
    """Where a BF16 GEMM launch's time goes (gcnn_gemm_study): the step's six GEMM
    shapes for a batch of --atoms atoms at H = 200, under the planner's plan and
    under every plan of its search space; and the update shape's time against K
    without split-K, fitted per tile width as fixed + per-64-wide-k-tile cost."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    import paper_2207_11333_gb300 as g
    plans = g.gemm_study(args.atoms, H, 0)
    shapes = {}
    for name in g.GEMM_SHAPES:
        rows = [r for r in plans if r["shape"] == name]
        own = next(r for r in rows if r["planner"])
        best = min(rows, key=lambda r: r["us"])
        pick = lambda r: {k: r[k] for k in ("BN", "ntiles", "splits", "cluster", "us")}
        shapes[name] = {"planner": pick(own), "fastest": pick(best), "plans_timed": len(rows),
                        "planner_over_fastest": own["us"] / best["us"]}
    sweep = g.gemm_study(args.atoms, H, 1)
    fits = {}
    for bn in sorted({r["BN"] for r in sweep}):
        pts = [(r["K"] / 64.0, r["us"]) for r in sweep if r["BN"] == bn and r["K"] >= 1024]
        x = np.array([p[0] for p in pts]); y = np.array([p[1] for p in pts])
        slope, icpt = np.polyfit(x, y, 1)
        mac_per_cycle = BM_ROWS * bn * 64 / (slope * 1e-6 * SM_CLOCK_HZ)
        fits[str(bn)] = {"us_per_k_tile": float(slope), "fixed_us": float(icpt),
                         "mac_per_cycle_per_sm": float(mac_per_cycle),
                         "times_us": {str(r["K"]): r["us"] for r in sweep if r["BN"] == bn}}
    print(json.dumps({"study": "gemm", "atoms": args.atoms, "hidden": H, "shapes": shapes,
                      "update_k_sweep_no_split": fits, "plans": plans,
                      "note": "us per launch, best of 5 replays of a 20-launch CUDA graph; k-tile = 64 of K; "
                              "MAC/cycle at 2070 MHz for a 128-row tile"}), flush=True)
    return 0


def serving_study(args):
    """The serving configuration alone: a student trained for a few hundred steps
    of the training workload serves Poisson traffic at every rate of
    --serve-rates for --serve-seconds each, beside the FP32 one-request-per-launch
    path; one JSON line."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    import paper_2207_11333_gb300 as g
    wl = Workload(g, 0, 1)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    loss_acc = torch.zeros(3, dtype=torch.float64, device="cuda")
    ctx = make_ctx(g, wl, args.precision)
    timed_steps(ctx, wl, args.steps, args.warmup, flush, loss_acc)
    trained = ctx.get_params()
    out = run_serving(g, ctx, wl.delta, trained, args)
    ctx.close()
    print(json.dumps({"study": "serving", "trained_steps": args.steps + args.warmup, **out}), flush=True)
    return 0


def run_ours(args):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_2207_11333_gb300 as g

    ddp = world > 1 or args.ddp
    if ddp and dist is None:    # --ddp at one process: the data-parallel path in a group of one
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{os.environ.get('MASTER_PORT', '29533')}",
                                rank=0, world_size=1)
    t_setup = time.perf_counter()
    wl = Workload(g, rank, world, ddp)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > 129 MB L2
    loss_acc = torch.zeros(3, dtype=torch.float64, device="cuda")
    log(f"[bench] setup {time.perf_counter() - t_setup:.1f}s, capacity N={wl.Nc} E={wl.Ec}, delta={wl.delta:.6f}")

    if ddp:
        return run_ddp(g, wl, args, world, rank, local, dist, flush, loss_acc)
    ctx = make_ctx(g, wl, args.precision)
    r = timed_steps(ctx, wl, args.steps, args.warmup, flush, loss_acc, dist, local)
    line = {"metric": METRIC, "value": r["value"], "unit": "graphs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * r["dev_s"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if args.precision == "bf16" else "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "graphs": N_TRAIN, "batch_graphs": BATCH, "hidden": H, "layers": L,
                       "head": "200-200-1", "precision": args.precision, "parallelism": f"replicas x{world}",
                       "gemms": "BF16 tcgen05, FP32 accumulate; aggregation, scalers, std, pooling, loss FP32"
                                if args.precision == "bf16" else "FP32 FFMA everywhere",
                       "l2": "256 MB buffer written between steps, outside the per-step CUDA events",
                       "wall_ms_per_step_incl_flush": 1e3 * r["wall_s"] / args.steps},
            "clocks": r["clocks"], "gpu_launches": r["kernels_per_step"] * args.steps}
    if not args.no_e2e:
        try:
            line["e2e"] = e2e_steps(g, ctx, wl, args.steps, loss_acc)
        except Exception as e:  # noqa: BLE001
            line["e2e"] = {"error": repr(e)}
    try:
        line.update(kernel_profile(g, wl, min(args.steps, 100), args.warmup, flush, loss_acc, args.precision))
    except Exception as e:  # noqa: BLE001
        line["roofline"] = {"error": repr(e)}
    ctx.check()
    if args.studies and world == 1:
        for key, fn in (("aggregate_large_batch", lambda: aggregate_large(g)),
                        ("recompute", lambda: recompute_study(g, args.precision)),
                        ("data_loading", lambda: loading_study(g)),
                        ("next_rows", lambda: variants_study(g, wl, flush, args.precision))):
            try:
                line[key] = fn()
            except Exception as e:  # noqa: BLE001
                line[key] = {"error": repr(e)}
    if args.serve_seconds > 0 and world == 1:
        try:
            trained = ctx.get_params()
            line["serving"] = run_serving(g, ctx, wl.delta, trained, args)
        except Exception as e:  # noqa: BLE001
            line["serving"] = {"error": repr(e)}
    ctx.close()
    if args.compare != "none" and args.compare != args.precision:
        c2 = make_ctx(g, wl, args.compare)
        r2 = timed_steps(c2, wl, args.steps, args.warmup, flush, loss_acc, dist)
        cmp = {"value": r2["value"], "unit": "graphs/s", "ms_per_step": 1e3 * r2["dev_s"] / args.steps,
               "precision": args.compare}
        try:
            prof = kernel_profile(g, wl, min(args.steps, 50), args.warmup, flush, loss_acc, args.compare)
            cmp["roofline"] = prof["roofline"]
            cmp["kernel_ms_per_step"] = prof["kernel_ms_per_step"]
            cmp["phase_us_per_step"] = prof["phase_us_per_step"]
        except Exception as e:  # noqa: BLE001
            cmp["roofline"] = {"error": repr(e)}
        c2.check()
        c2.close()
        line[f"{args.compare}_path"] = cmp
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            os.environ.setdefault("OMP_NUM_THREADS", str(len(os.sched_getaffinity(0))))
            line["cpu_baseline"] = oracle_graphs_per_s(wl.path, wl.order, budget_s=args.cpu_seconds)
            line["cpu_baseline"]["single_thread"] = oracle_single_thread(wl.path, wl.order, args.cpu_seconds / 2)
        except Exception as e:  # noqa: BLE001
            line["cpu_baseline"] = {"error": repr(e)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_ddp(g, wl, args, world, rank, local, dist, flush, loss_acc):
    """The bench line of the data-parallel step: world processes, one GPU each,
    128 graphs per process and step, gradients all-reduced every step."""
    import torch
    prec = g.PREC_BF16 if args.precision == "bf16" else g.PREC_FP32
    ctx = g.Context(g.make_config(H, L, BATCH, wl.Nc, wl.Ec, delta=wl.delta, precision=prec))
    ctx.set_params(synth.init_params(SEED_STUDENT, H, L))
    r = timed_ddp_steps(g, ctx, wl, args.steps, args.warmup, flush, loss_acc, dist, local)
    line = {"metric": METRIC, "value": r["value"], "unit": "graphs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * r["dev_s"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if args.precision == "bf16" else "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "graphs": N_TRAIN, "batch_graphs_per_gpu": BATCH, "hidden": H,
                       "layers": L, "head": "200-200-1", "precision": args.precision,
                       "parallelism": f"ddp x{world}: gradient all-reduce (NCCL) per layer bucket, overlapped "
                                      "with the backward; forward + backward from one captured graph, the "
                                      "all-reduces and AdamW launched after it",
                       "l2": "256 MB buffer written between steps, outside the per-step CUDA events",
                       "wall_ms_per_step_incl_flush": 1e3 * r["wall_s"] / args.steps},
            "clocks": r["clocks"], "gpu_launches": r["kernels_per_step"] * args.steps}
    if not args.no_e2e:
        try:
            sh = g.Store(wl.path)           # host-resident twin: pinned staging + H2D per step
            sh.set_targets(wl.y)
            e = timed_ddp_steps(g, ctx, wl, args.steps, args.warmup, flush, loss_acc, dist, None, store=sh, e2e=True)
            line["e2e"] = {"value": e["value"], "unit": "graphs/s", "h2d_bytes_per_step": e["h2d_bytes_per_step"],
                           "d2h_bytes_per_step": 24,
                           "path": "DataParallelTrainer from a host store; every step's loss read back"}
        except Exception as ex:  # noqa: BLE001
            line["e2e"] = {"error": repr(ex)}
    ctx.check()
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    dist.barrier()
    dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "bf16"], default="bf16",
                    help="GEMM precision of the measured path (bf16: tensor cores, FP32 accumulate)")
    ap.add_argument("--compare", choices=["none", "fp32", "bf16"], default="fp32",
                    help="also time this path on the same workload (default: the plain FP32 path)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--ddp", action="store_true",
                    help="data-parallel steps (gradient all-reduce) also at one GPU; always on for N > 1")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=150.0,
                    help="host-time budget of the reference arm's warm-up and timed steps")
    ap.add_argument("--serve-seconds", type=float, default=3.0,
                    help="seconds of Poisson load per arrival rate for the serving measurement (0: skip)")
    ap.add_argument("--serve-rates", default="50,200,500,1000,2000", help="arrival rates, requests/s")
    ap.add_argument("--serve-slots", type=int, default=4, help="server slots (batches in flight)")
    ap.add_argument("--baseline-seconds", type=float, default=20.0,
                    help="seconds per rate of the one-request-per-launch FP32 baseline (at most --serve-seconds)")
    ap.add_argument("--study", choices=["none", "precision", "aggregate", "loading", "serving", "gemm"],
                    default="none",
                    help="precision: train FP32 and BF16 for --epochs and compare held-out MAE; aggregate: the "
                         "aggregation operators alone on --molecules molecules, --reps timed launches each "
                         "(no bench line)")
    ap.add_argument("--molecules", type=int, default=60_000, help="batch of the aggregation study")
    ap.add_argument("--atoms", type=int, default=2304, help="batch atoms of the GEMM study (128 molecules of 18)")
    ap.add_argument("--reps", type=int, default=5, help="timed launches per operator in the aggregation study")
    ap.add_argument("--epochs", type=int, default=10)
    ap.add_argument("--seeds", type=int, default=1, help="precision study: initial parameters and orders to repeat over")
    ap.add_argument("--lr", type=float, default=1e-4, help="learning rate of the precision study")
    ap.add_argument("--no-studies", dest="studies", action="store_false",
                    help="skip the large-batch aggregation and recompute measurements")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.study == "precision":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        import paper_2207_11333_gb300 as g
        print(json.dumps({"study": "precision", **precision_study(g, args.epochs, args.lr, args.seeds)}), flush=True)
        return 0
    if args.study == "loading":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        import paper_2207_11333_gb300 as g
        print(json.dumps({"study": "loading", **loading_study(g)}), flush=True)
        return 0
    if args.study == "serving":
        return serving_study(args)
    if args.study == "gemm":
        return gemm_study(args)
    if args.study == "aggregate":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        import paper_2207_11333_gb300 as g
        print(json.dumps({"study": "aggregate", **aggregate_large(g, args.reps, args.molecules)}), flush=True)
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
