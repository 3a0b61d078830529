"""Distributed data parallelism (Sec. 4, Fig. 4) through the library on one GPU.

- Shards run one after another: for each process's share of a global batch the
  context's loss gradient is scaled by that share (gcnn_set_loss_scale), and
  the sum of the shards' gradients equals the whole batch's gradient from the
  library (FP32 summation order only) and the FP64 oracle's (the gradient
  gate), with the node-level head and bond features so that both scales act.
- DataParallelTrainer in a process group of one over NCCL: the bucketed
  all-reduce on its own stream, ordered after gcnn_grad_wait, and the AdamW
  step after it give the same parameters, bit for bit, as the plain eager
  steps, with the forward + backward from one captured graph and eager.
- Two processes share the GPU with gloo (the all-reduce goes through host
  memory; no kernel waits on another process): both end with identical
  parameters, which match the oracle's steps on the whole global batches.
"""
import dataclasses
import os
import socket

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_common import context, write_both
from helpers import FP32_GRAD_TOL, Gates, rel_norm

pytestmark = pytest.mark.gpu

H, L, F, W = 32, 2, 4, 0.7


def _workload(G=60):
    d = oracle.Dims(H=H, L=L, F=F, NH=1, node_weight=W)
    gs = synth.molecules_uniform(81, G, 4, 30)
    gs.y = synth.uniform_targets(82, 0, G, 1.0, 10.0)
    gs.ynode = synth.uniform(83, 0, gs.n_nodes, -1.0, 1.0).astype(np.float32)
    gs.eattr = synth.bond_features(84, gs, F, -1.0, 1.0)
    p = synth.init_params(85, H, L, F=F)
    pad = np.zeros((p.size + 3) // 4 * 4 - p.size, np.float32)
    nh = synth.init_params(86, H, 1)[-(H * H + 2 * H + 1):]
    return d, gs, np.concatenate([p, pad, nh])


def _ctx(gs, delta, precision=0):
    return context(H, L, gs.n_graphs, gs.n_nodes, gs.n_edges, delta, precision=precision, F=F, node_head=1,
                   node_weight=W)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_sequential_shards_sum_to_the_whole_batch(tmp_path):
    import paper_2207_11333_gb300 as g
    from paper_2207_11333_gb300.ddp import ShardedSampler
    d, gs, p = _workload()
    path, ost = write_both(gs, str(tmp_path))
    st = g.Store(path)
    delta = st.delta()
    counts = np.diff(gs.node_ptr)
    world, B = 3, 16
    gates = Gates("shards run one after another")
    ctx = _ctx(gs, delta)
    ctx.set_params(p)
    for step in range(2):
        samplers = [ShardedSampler(gs.n_graphs, B, world, r, seed=9, node_counts=counts) for r in range(world)]
        total = np.zeros(ctx.n_params)
        for r in range(world):
            sh = samplers[r].shard(step)
            b = ctx.collate(st, sh.ids)
            ctx.set_loss_scale(*sh.scales(r))
            ctx.forward(b, train=True)
            ctx.backward(b)
            total += ctx.get_grads().astype(np.float64)
        glob = samplers[0].order[step * world * B:(step + 1) * world * B]
        ctx.set_loss_scale(1.0, 1.0)
        b = ctx.collate(st, glob)
        ctx.forward(b, train=True)
        ctx.backward(b)
        whole = ctx.get_grads()
        _, ograd, _, _ = oracle.backward(d, p.astype(np.float64), oracle.collate(ost, glob, delta))
        gates.check(f"shards vs whole, step {step}", total, whole, 1e-5)
        gv, ov = oracle.split_params(d, total), oracle.split_params(d, ograd)
        for k in ov:
            gates.check(f"{k} s{step}", gv[k], ov[k], FP32_GRAD_TOL)
    ctx.check()
    gates.assert_all()


def test_trainer_in_a_group_of_one_over_nccl(tmp_path):
    import torch.distributed as dist

    import paper_2207_11333_gb300 as g
    from paper_2207_11333_gb300.ddp import DataParallelTrainer, ShardedSampler
    d, gs, p = _workload()
    path, _ = write_both(gs, str(tmp_path))
    st = g.Store(path)
    delta = st.delta()
    counts = np.diff(gs.node_ptr)
    steps, lr = 3, 1e-3
    plain = _ctx(gs, delta, precision=1)
    plain.set_params(p)
    sampler = ShardedSampler(gs.n_graphs, 16, 1, 0, seed=4, node_counts=counts)
    for s in range(steps):
        b = plain.collate(st, sampler.shard(s).ids)
        plain.forward(b, train=True)
        plain.backward(b)
        plain.step(lr)
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{_free_port()}", rank=0, world_size=1)
    try:
        for captured in (True, False):      # one graph per forward + backward, or eager calls
            ctx = _ctx(gs, delta, precision=1)
            ctx.set_params(p)
            tr = DataParallelTrainer(ctx, st, sampler, captured=captured)
            assert tr.dist is not None and tr.comm is not None and tr.captured == captured
            for s in range(steps):
                tr.step(s, lr)
            torch.cuda.synchronize()
            assert np.array_equal(ctx.get_params(), plain.get_params()), captured
            ctx.check()
            ctx.close()
    finally:
        dist.destroy_process_group()


def test_forward_backward_graph_then_step_equals_train_step(tmp_path):
    """gcnn_forward_backward (captured, bucket events as external graph nodes)
    followed by gcnn_step gives the parameters of gcnn_train_step bit for bit,
    FP32 and BF16, and a stream can wait on every bucket afterwards."""
    import paper_2207_11333_gb300 as g
    d, gs, p = _workload()
    path, _ = write_both(gs, str(tmp_path))
    st = g.Store(path)
    delta = st.delta()
    for precision in (0, 1):
        a, b2 = _ctx(gs, delta, precision), _ctx(gs, delta, precision)
        a.set_params(p)
        b2.set_params(p)
        side = torch.cuda.Stream()
        for k in range(3):
            ids = np.random.default_rng(k).permutation(gs.n_graphs)[:40]
            a.train_step(a.collate(st, ids), 1e-3)
            bb = b2.collate(st, ids)
            b2.forward_backward(bb)
            for bucket in range(len(b2.grad_buckets())):
                b2.grad_wait(bucket, side)
            torch.cuda.current_stream().wait_stream(side)
            b2.step(1e-3)
        torch.cuda.synchronize()
        assert np.array_equal(a.get_params(), b2.get_params()), precision
        a.check()
        b2.check()


def _rank_main(rank, world, port, path, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import paper_2207_11333_gb300 as g
        from paper_2207_11333_gb300.ddp import DataParallelTrainer, ShardedSampler
        d, gs, p = _workload()
        st = g.Store(path)
        delta = st.delta()
        counts = np.diff(gs.node_ptr)
        sampler = ShardedSampler(gs.n_graphs, 12, world, rank, seed=13, node_counts=counts)
        ctx = _ctx(gs, delta)
        ctx.set_params(p)
        tr = DataParallelTrainer(ctx, st, sampler)
        for s in range(len(sampler)):
            tr.step(s, 1e-3)
        ctx.check()
        theta = torch.from_numpy(ctx.get_params())
        other = theta.clone()
        dist.broadcast(other, src=0)
        out = {"rank": rank, "spread": float(torch.max(torch.abs(theta - other))), "steps": len(sampler)}
        if rank == 0:       # the oracle on each whole global batch
            ost = oracle.read_store(path)
            th = p.astype(np.float64)
            m, v = np.zeros_like(th), np.zeros_like(th)
            for s in range(len(sampler)):
                glob = sampler.order[s * world * 12:(s + 1) * world * 12]
                _, grad, _, _ = oracle.backward(d, th, oracle.collate(ost, glob, delta))
                oracle.adam(th, grad, m, v, s + 1, lr=1e-3)
            out["change"] = rel_norm(theta.numpy().astype(np.float64) - p, th - p)
            out["theta"] = rel_norm(theta.numpy(), th)
        q.put(out)
    finally:
        dist.destroy_process_group()


def test_two_processes_share_the_gpu_over_gloo(tmp_path):
    import torch.multiprocessing as mp
    d, gs, p = _workload()
    path, _ = write_both(gs, str(tmp_path))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, path, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = {}
    for _ in procs:
        o = q.get(timeout=600)
        res[o["rank"]] = o
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    assert res[0]["steps"] == 3                     # 60 graphs, 2 x 12 per step, a 12-graph tail
    assert res[0]["spread"] == 0.0 and res[1]["spread"] == 0.0
    assert res[0]["change"] < 1e-3, res[0]
    assert res[0]["theta"] < 1e-5, res[0]
