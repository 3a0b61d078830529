"""Distributed data parallelism (Sec. 4, Fig. 4) on the host: two gloo ranks run
the package's DataParallelTrainer (sharded sampler, loss scales, bucketed
all-reduce, optimizer step) over a context-shaped object backed by the FP64
oracle.  After the exchange every rank holds the gradient of the whole
global batch (as one process collating all of the step's graphs would compute
it), both ranks' parameters stay identical, the shards of an epoch are
disjoint and cover it, and the buckets cover the flat gradient buffer once.
The model has the node-level head and bond features, so both loss scales
(graphs and atoms) matter; the global batches split unevenly."""
import dataclasses
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth
from paper_2207_11333_gb300.ddp import DataParallelTrainer, ShardedSampler

G_ALL, LOCAL_BATCH, H, L, F = 27, 5, 8, 2, 4


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _data():
    d = oracle.Dims(H=H, L=L, F=F, NH=1, node_weight=0.7)
    gs = synth.molecules_uniform(71, G_ALL, 4, 22)
    gs.y = synth.uniform_targets(72, 0, G_ALL, 1.0, 10.0)
    gs.ynode = synth.uniform(73, 0, gs.n_nodes, -1.0, 1.0).astype(np.float32)
    gs.eattr = synth.bond_features(74, gs, F, -1.0, 1.0)
    st = oracle.store_from_arrays(gs.node_ptr, gs.edge_ptr, gs.types, gs.edges, gs.y, gs.eattr, gs.ynode)
    p = synth.init_params(75, H, L, F=F)
    pad = np.zeros((p.size + 3) // 4 * 4 - p.size, np.float32)
    nh = synth.init_params(76, H, 1)[-(H * H + 2 * H + 1):]
    p = np.concatenate([p, pad, nh]).astype(np.float64)
    assert p.size == oracle.param_count(d)
    return d, gs, st, oracle.delta_of(st), p


def buckets_of(d, P):
    """The library's bucket layout: layers, then head/bond rows/node head, then the embedding."""
    lb, ls = d.T * d.H, 18 * d.H * d.H + 2 * d.H
    le = lb + d.L * ls
    return [(lb + l * ls, ls) for l in range(d.L)] + [(le, P - le), (0, lb)]


class OracleContext:
    """The context interface DataParallelTrainer drives, computed by the FP64
    oracle on the host: the loss scales multiply the graph-level loss gradient
    (through dpred) and the node-level loss weight."""

    def __init__(self, d, st, delta, params):
        self.d, self.st, self.delta = d, st, delta
        self.p = params.copy()
        self.m, self.v, self.t = np.zeros_like(self.p), np.zeros_like(self.p), 0
        self.g = torch.zeros(self.p.size, dtype=torch.float64)
        self.scale = (1.0, 1.0)

    def collate(self, store, ids):
        return oracle.collate(self.st, ids, self.delta)

    def set_loss_scale(self, graph_scale, node_scale=1.0):
        self.scale = (graph_scale, node_scale)

    def forward(self, b, train=True):
        self.b = b

    def backward(self, b, dpred=None, loss_accum=None):
        pred = oracle.forward(self.d, self.p, b)
        dp = self.scale[0] * 2.0 * (pred - b.y.astype(np.float64)) / b.G
        d = dataclasses.replace(self.d, node_weight=self.d.node_weight * self.scale[1])
        _, grad, _, _ = oracle.backward(d, self.p, b, dpred=dp)
        self.g.copy_(torch.from_numpy(grad))

    def grad_buckets(self):
        return buckets_of(self.d, self.p.size)

    def grad_wait(self, bucket, stream):
        pass

    def grads_tensor(self):
        return self.g

    def step(self, lr):
        self.t += 1
        oracle.adam(self.p, self.g.numpy().copy(), self.m, self.v, self.t, lr=lr)


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        d, gs, st, delta, p = _data()
        counts = np.diff(gs.node_ptr)
        sampler = ShardedSampler(G_ALL, LOCAL_BATCH, world, rank, seed=11, node_counts=counts)
        ctx = OracleContext(d, st, delta, p)
        tr = DataParallelTrainer(ctx, None, sampler)
        ref = OracleContext(d, st, delta, p)      # one process on each whole global batch
        errs, mine = [], []
        for s in range(len(sampler)):
            sh = tr.step(s, 1e-3)
            mine.append(sh.ids.tolist())
            glob = sampler.order[s * world * LOCAL_BATCH:(s + 1) * world * LOCAL_BATCH]
            b = ref.collate(None, glob)
            ref.backward(b)
            ref.step(1e-3)
            errs.append((float(np.linalg.norm(ctx.g.numpy() - ref.g.numpy()) / np.linalg.norm(ref.g.numpy())),
                         float(np.max(np.abs(ctx.p - ref.p)))))
        theta = torch.from_numpy(ctx.p.copy())
        other = theta.clone()
        dist.broadcast(other, src=0)
        q.put((rank, errs, mine, float(torch.max(torch.abs(theta - other))), len(sampler)))
    finally:
        dist.destroy_process_group()


def test_two_rank_data_parallel_steps_match_one_process():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = dict()
    for _ in procs:
        r, errs, mine, spread, steps = q.get(timeout=300)
        res[r] = (errs, mine, spread, steps)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    steps = res[0][3]
    assert steps == 3                               # 27 graphs, 2 x 5 per step: 2 full steps + a 7-graph step
    for r in (0, 1):
        errs, mine, spread, _ = res[r]
        assert spread == 0.0                        # every rank applies the same update
        for g_err, p_err in errs:
            assert g_err < 1e-13 and p_err < 1e-13, errs
    seen = sorted(i for r in (0, 1) for step in res[r][1] for i in step)
    assert seen == sorted(set(seen)) and len(seen) == G_ALL    # disjoint, and the whole epoch
    sizes = [len(step) for step in res[0][1]] + [len(step) for step in res[1][1]]
    assert sorted(sizes) == [3, 4, 5, 5, 5, 5]                 # the last global batch splits 4 + 3


def test_sampler_and_buckets_on_the_host():
    d, gs, st, delta, p = _data()
    b = buckets_of(d, p.size)
    cover = np.zeros(p.size, np.int64)
    for o, c in b:
        cover[o:o + c] += 1
    assert np.all(cover == 1)
    counts = np.diff(gs.node_ptr)
    s = [ShardedSampler(G_ALL, 4, 3, r, seed=5, node_counts=counts) for r in range(3)]
    assert len(s[0]) == 3                    # 12 per step: 2 full steps, a 3-graph tail
    for k in range(len(s[0])):
        shards = [x.shard(k) for x in s]
        assert shards[0].graphs == shards[1].graphs == shards[2].graphs
        assert [len(x.ids) for x in shards] == shards[0].graphs
        assert abs(sum(x.scales(r)[0] for r, x in enumerate(shards)) - 1.0) < 1e-15
        assert abs(sum(x.scales(r)[1] for r, x in enumerate(shards)) - 1.0) < 1e-15
        assert [int(counts[x.ids].sum()) for x in shards] == shards[0].atoms
    s2 = ShardedSampler(2, 4, 3, 0, seed=5)
    assert len(s2) == 0                      # a tail of fewer graphs than processes is dropped
    s[0].set_epoch(1)
    assert not np.array_equal(s[0].order, s[1].order)


def _post_and_exit(q, msg):
    """Deliver msg, then end the process without the process group's shutdown
    (which would wait on the departed peer)."""
    q.put(msg)
    q.close()
    q.join_thread()
    os._exit(0)


DROP_TIMEOUT_S = 4.0


def _dropout_main(rank, world, port, q, how):
    import datetime
    import time
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=DROP_TIMEOUT_S))
    d, gs, st, delta, p = _data()
    sampler = ShardedSampler(G_ALL, LOCAL_BATCH, world, rank, seed=11, node_counts=np.diff(gs.node_ptr))
    ctx = OracleContext(d, st, delta, p)
    tr = DataParallelTrainer(ctx, None, sampler)
    tr.step(0, 1e-3)
    if rank == 1:                       # leaves between steps, nothing in flight
        if how == "stalls":             # alive, but never joins the next exchange
            time.sleep(3 * DROP_TIMEOUT_S)
        _post_and_exit(q, (1, "left", 0.0, 0.0, ""))
    before = ctx.p.copy()
    t0 = time.monotonic()
    try:
        tr.step(1, 1e-3)
        msg = (0, "no error", time.monotonic() - t0, 0.0, "")
    except RuntimeError as e:
        msg = (0, "error", time.monotonic() - t0, float(np.max(np.abs(ctx.p - before))), str(e)[:200])
    _post_and_exit(q, msg)


@pytest.mark.parametrize("how", ["exits", "stalls"])
def test_rank_that_drops_out_fails_the_next_exchange_on_the_host(how):
    """A rank leaves between steps (fault injected on the host): it exits, or it
    stays alive and never joins the next exchange.  The other rank's next step
    raises on the host, at once when the peer's connection closes and after the
    process group's timeout when it stalls, and leaves its parameters as they
    were: the optimizer step never runs on a partial sum."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dropout_main, args=(r, 2, port, q, how)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = {}
    for _ in procs:
        r, what, secs, moved, why = q.get(timeout=120)
        res[r] = (what, secs, moved, why)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    assert res[1][0] == "left"
    what, secs, moved, why = res[0]
    assert what == "error", res[0]
    assert secs < (1.0 if how == "exits" else 3 * DROP_TIMEOUT_S), res[0]
    if how == "stalls":
        assert secs >= 0.9 * DROP_TIMEOUT_S, res[0]
    assert moved == 0.0
