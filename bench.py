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


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dataset():
    gs = synth.molecules_lognormal(SEED_DATA, N_TRAIN + N_HELDOUT)
    return gs


def epoch_order(rank: int = 0) -> np.ndarray:
    return np.random.default_rng(SEED_ORDER + 1000 * rank).permutation(N_TRAIN).astype(np.int64)


def gemm_flops(n_nodes: int) -> float:
    """Algorithmic FLOPs of the step's dense GEMMs for a batch of n_nodes (all layers, fwd + bwd)."""
    per_layer = 2.0 * n_nodes * (H * 2 * H + 16 * H * H)          # forward: message, update
    per_layer += 2.0 * n_nodes * (16 * H * H + 3 * H * 5 * H + H * 2 * H + 3 * H * H)  # dW_U, dagg, dW_M, dx
    return L * per_layer


def agg_fwd_bytes(n_nodes: int, n_edges: int) -> float:
    """Compulsory bytes of one aggregation launch: P and Q rows read once, 5H written, CSR read."""
    return n_nodes * (2 * H + 5 * H) * 4.0 + (n_nodes + 1 + n_edges) * 4.0


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
def oracle_graphs_per_s(path: str, order: np.ndarray, budget_s: float, max_graphs: int = BATCH):
    """Time the FP64 oracle's fwd + bwd + Adam on a bounded sample of the workload."""
    import oracle
    cores = len(os.sched_getaffinity(0))
    ost = oracle.read_store(path)
    ost.y = synth.uniform_targets(SEED_DATA + 7, 0, len(ost.y), 1.0, 10.0)   # targets independent of the GPU
    d = oracle.Dims(H=H, L=L)
    p = synth.init_params(SEED_STUDENT, H, L).astype(np.float64)
    delta = oracle.delta_of(ost, order[:2048])

    def run(ids):
        b = oracle.collate(ost, ids, delta)
        t0 = time.perf_counter()
        loss, grad, _, _ = oracle.backward(d, p, b)
        th = p.copy()
        oracle.adam(th, grad, np.zeros_like(p), np.zeros_like(p), 1, lr=LR)
        return time.perf_counter() - t0

    t_cal = run(order[:4])
    per_graph = max(t_cal / 4, 1e-6)
    n = int(max(4, min(max_graphs, budget_s / per_graph)))
    t = run(order[4:4 + n])
    return {"value": n / t, "unit": "graphs/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} graphs of the workload (one batch), FP64 fwd+bwd+AdamW, {t:.1f} s, "
                      f"OpenMP over nodes on {cores} host cores"}


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
    budget = 150.0
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

    t_setup = time.perf_counter()
    gs = dataset()
    tmp = tempfile.mkdtemp(prefix="gcnn_bench_")
    path = os.path.join(tmp, "train.gcnn")
    synth.write_store(path, gs)
    st = g.Store(path)
    st.to_device()
    delta = st.delta(np.arange(N_TRAIN))
    y = make_targets(g, st, delta, N_TRAIN + N_HELDOUT)
    st.set_targets(y)
    order = epoch_order(rank)
    nb = (N_TRAIN + BATCH - 1) // BATCH
    sizes = [st.batch_size(order[i * BATCH:(i + 1) * BATCH]) for i in range(nb)]
    Nc = (max(s[0] for s in sizes) + 255) // 256 * 256
    Ec = (max(s[1] for s in sizes) + 511) // 512 * 512
    prec = g.PREC_BF16 if args.precision == "bf16" else g.PREC_FP32
    ctx = g.Context(g.make_config(H, L, BATCH, Nc, Ec, delta=delta, precision=prec))
    ctx.set_params(synth.init_params(SEED_STUDENT, H, L))
    ctx.set_order(st, order)
    loss_acc = torch.zeros(3, dtype=torch.float64, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > 129 MB L2
    log(f"[bench] setup {time.perf_counter() - t_setup:.1f}s, capacity N={Nc} E={Ec}, delta={delta:.6f}")

    def batch_at(k):
        i = k % nb
        return ctx.collate_range(st, i * BATCH, min(BATCH, N_TRAIN - i * BATCH))

    for k in range(args.warmup):
        ctx.train_step(batch_at(k), LR, loss_acc)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    graphs = 0
    torch.cuda.nvtx.range_push("timed")
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        evs[k][0].record()
        b = batch_at(args.warmup + k)
        ctx.train_step(b, LR, loss_acc)
        evs[k][1].record()
        graphs += b.n_graphs
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    torch.cuda.nvtx.range_pop()
    clocks = sampler.stop()
    dev_ms = sum(a.elapsed_time(b) for a, b in evs)
    kernels_per_step = ctx.step_kernel_count() + 2
    if dist:
        tt = torch.tensor([dev_ms / 1e3, float(graphs)], dtype=torch.float64, device="cuda")
        tmax = tt[:1].clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        gsum = tt[1:].clone()
        dist.all_reduce(gsum, op=dist.ReduceOp.SUM)
        t_dev, total_graphs = float(tmax.item()), float(gsum.item())
    else:
        t_dev, total_graphs = dev_ms / 1e3, float(graphs)
    value = total_graphs / t_dev
    line = {"metric": METRIC, "value": value, "unit": "graphs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if prec else "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "graphs": N_TRAIN, "batch_graphs": BATCH, "hidden": H, "layers": L,
                       "head": "200-200-1", "precision": args.precision, "parallelism": f"replicas x{world}",
                       "l2": "256 MB buffer written between steps, outside the per-step CUDA events",
                       "wall_ms_per_step_incl_flush": 1e3 * wall / args.steps},
            "clocks": clocks, "gpu_launches": kernels_per_step * args.steps}

    # end to end through the public API from host memory
    if not args.no_e2e:
        try:
            sh = g.Store(path)          # host-resident twin: collation stages through pinned memory
            sh.set_targets(y)
            pinned = torch.zeros(3, dtype=torch.float64).pin_memory()
            k_e2e = args.steps
            h2d = 0
            for k in range(3):
                i = k % nb
                ctx.train_step(ctx.collate(sh, order[i * BATCH:(i + 1) * BATCH]), LR, loss_acc)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            n_e2e = 0
            for k in range(k_e2e):
                i = (args.warmup + k) % nb
                ids = order[i * BATCH:(i + 1) * BATCH]
                b = ctx.collate(sh, ids)
                ctx.train_step(b, LR, loss_acc)
                pinned.copy_(loss_acc, non_blocking=True)
                torch.cuda.current_stream().synchronize()
                _ = float(pinned[0])
                n_e2e += b.n_graphs
                h2d += 16 * (b.n_graphs + 1) + 4 * b.n_graphs + b.n_nodes + 2 * b.n_edges
            dt = time.perf_counter() - t0
            line["e2e"] = {"value": n_e2e / dt, "unit": "graphs/s", "h2d_bytes_per_step": h2d / k_e2e,
                           "d2h_bytes_per_step": 24, "steps": k_e2e,
                           "path": "gcnn_collate from a host store (pinned staging, one H2D) + gcnn_train_step "
                                   "+ loss read back each step"}
        except Exception as e:  # noqa: BLE001
            line["e2e"] = {"error": repr(e)}

    # kernel-level timing: the same steps eagerly, CUDA events around every launch
    try:
        ctx.profile(True)
        ctx.profile_read()
        n_prof = min(args.steps, 100)
        flops = 0.0
        agg_bytes = 0.0
        for k in range(n_prof):
            flush.zero_()
            b = batch_at(args.warmup + k)
            ctx.train_step(b, LR, loss_acc)
            flops += gemm_flops(b.n_nodes)
            agg_bytes += L * agg_fwd_bytes(b.n_nodes, b.n_edges)
        ph = ctx.profile_read()
        ctx.profile(False)
        line["phases_ms_per_step"] = {k: v[0] / n_prof for k, v in ph.items()}
        gemm_ms = ph["gemm"][0]
        sm_mhz = 2070.0
        peak_alu = SM_COUNT * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
        achieved = flops / (gemm_ms / 1e3) / 1e12
        line["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak_alu, "unit": "TFLOP/s",
                            "frac": achieved / peak_alu, "traffic": None,
                            "kernel": "sgemm_kernel + splitk_reduce (all dense GEMMs of the step, FP32 FFMA)",
                            "peak_source": "152 SMs x 128 FP32 lanes x 2 FLOP x 2070 MHz (derived; no measured FP32 peak)"}
        agg_ms = ph["agg_fwd"][0]
        hbm, hbm_src = measured_hbm()
        a_gbs = agg_bytes / (agg_ms / 1e3) / 1e9
        line["roofline_aggregate"] = {"bound": "hbm", "achieved": a_gbs, "peak": hbm, "unit": "GB/s",
                                      "frac": a_gbs / hbm, "traffic": None, "peak_source": hbm_src,
                                      "note": "batch working set fits in L2; the HBM figure needs a >L2 batch"}
    except Exception as e:  # noqa: BLE001
        line["roofline"] = {"error": repr(e)}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            os.environ.setdefault("OMP_NUM_THREADS", str(len(os.sched_getaffinity(0))))
            line["cpu_baseline"] = oracle_graphs_per_s(path, order, budget_s=args.cpu_seconds)
        except Exception as e:  # noqa: BLE001
            line["cpu_baseline"] = {"error": repr(e)}
    ctx.check()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "bf16"], default="fp32")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
