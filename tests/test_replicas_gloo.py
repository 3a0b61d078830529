"""Multi-rank semantics on CPU (gloo, world size 2): each rank takes a disjoint shard
of the epoch order, and the count-weighted all-reduced shard gradients equal the
whole batch's gradient (the data-parallel identity the paper's DDP relies on).
The GPU path runs one replica per GPU with no data-path collective."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def shard(order, rank, world):
    return order[rank::world]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    H, L = 8, 2
    d = oracle.Dims(H=H, L=L)
    gs = synth.molecules_uniform(1, 24, 5, 20)
    gs.y = synth.uniform_targets(2, 0, 24, 1, 10)
    st = oracle.store_from_arrays(gs.node_ptr, gs.edge_ptr, gs.types, gs.edges, gs.y)
    delta = oracle.delta_of(st)
    order = np.random.default_rng(11).permutation(24)
    mine = shard(order, rank, world)
    p = synth.init_params(3, H, L).astype(np.float64)
    _, grad, _, _ = oracle.backward(d, p, oracle.collate(st, mine, delta))
    g = torch.from_numpy(grad * len(mine))
    dist.all_reduce(g)
    seen = torch.zeros(24, dtype=torch.int64)
    seen[torch.from_numpy(mine)] = 1
    dist.all_reduce(seen)
    if rank == 0:
        _, full, _, _ = oracle.backward(d, p, oracle.collate(st, order, delta))
        out.put((float(np.linalg.norm(g.numpy() / 24 - full) / np.linalg.norm(full)), seen.tolist()))
    dist.destroy_process_group()


def test_two_rank_shards_and_gradient_identity():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    err, seen = q.get(timeout=240)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    assert seen == [1] * 24          # disjoint and complete
    assert err < 1e-13
