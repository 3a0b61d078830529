"""Distributed data parallelism of the training step (Sec. 4, Fig. 4).

Every process holds a full replica of the model (one gcnn context on its own
GPU) and trains on its own graphs; before every optimizer step the processes
sum their gradients with an all-reduce, so every replica applies the same
update.  The library computes and applies; this module only arranges the data
partition and the exchange, with torch.distributed as the communicator (NCCL
across GPUs, gloo on the host):

- ShardedSampler: one seeded order of the training graphs per epoch, the same
  on every process; global step k takes world * local_batch consecutive
  graphs of that order and process r its r-th share of them (Sec. 4: each
  process reads its own portion of the data).
- DataParallelTrainer: per step, the process's share is collated, its loss
  gradient scaled by its share of the step's graphs (and atoms, for the
  node-level loss), the forward and backward launched (one captured graph),
  and each gradient bucket (one per
  conv layer, then the head and the embedding) all-reduced on a separate
  stream as soon as the library reports it final (gcnn_grad_wait), while the
  backward of the layers below still runs.  The optimizer step then waits for
  the last bucket.  The sum over processes of the scaled gradients is the
  gradient of the whole step's mean loss, as if one process had collated all
  of the step's graphs.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Shard:
    ids: np.ndarray          # this process's graph ids for the step
    graphs: list[int]        # graphs of every process for the step
    atoms: list[int]         # atoms of every process for the step

    def scales(self, rank: int) -> tuple[float, float]:
        """(graph_scale, node_scale) of process `rank`: its share of the step's
        graphs and atoms."""
        g, n = sum(self.graphs), sum(self.atoms)
        return (self.graphs[rank] / g if g else 0.0, self.atoms[rank] / n if n else 0.0)


class ShardedSampler:
    """Seeded epoch order split into global batches of world * local_batch graphs.

    Global step k of an epoch covers order[k W B : (k + 1) W B]; process r takes
    the r-th of W near-equal consecutive pieces of it.  A final global batch with
    fewer than W graphs is dropped, so every process has at least one graph in
    every step.  node_counts (atoms per graph of the whole set) give every
    process's atom count without communication.
    """

    def __init__(self, n_graphs: int, local_batch: int, world: int, rank: int, seed: int,
                 node_counts: np.ndarray | None = None):
        if not (0 <= rank < world) or local_batch < 1 or n_graphs < 1:
            raise ValueError("bad sampler arguments")
        self.n, self.B, self.W, self.rank, self.seed = n_graphs, local_batch, world, rank, seed
        self.node_counts = None if node_counts is None else np.asarray(node_counts, np.int64)
        self.set_epoch(0)

    def set_epoch(self, epoch: int) -> None:
        self.epoch = epoch
        self.order = np.random.default_rng([self.seed, epoch]).permutation(self.n).astype(np.int64)

    def __len__(self) -> int:
        gb = self.W * self.B
        full, tail = divmod(self.n, gb)
        return full + (1 if tail >= self.W else 0)

    def shard(self, step: int) -> Shard:
        if not 0 <= step < len(self):
            raise IndexError(step)
        gb = self.W * self.B
        glob = self.order[step * gb:(step + 1) * gb]
        pieces = np.array_split(glob, self.W)
        atoms = [int(self.node_counts[p].sum()) if self.node_counts is not None else 0 for p in pieces]
        return Shard(np.ascontiguousarray(pieces[self.rank]), [len(p) for p in pieces], atoms)


class DataParallelTrainer:
    """One data-parallel training step per call (forward, backward, gradient
    all-reduce by buckets, AdamW) on a context whose stream is torch's current
    stream.

    ctx: a paper_2207_11333_gb300.Context (or an object with the same
    collate / set_loss_scale / forward / backward / grad_buckets / grad_wait /
    grads_tensor / step methods); group: a torch.distributed process group (the
    default group when None; a single process when torch.distributed is not
    initialised).
    """

    def __init__(self, ctx, store, sampler: ShardedSampler, group=None, captured: bool = True):
        import torch.distributed as dist
        self.ctx, self.store, self.sampler, self.group = ctx, store, sampler, group
        # forward + backward from one captured graph (gcnn_forward_backward)
        # when the context offers it, else the eager calls
        self.captured = captured and hasattr(ctx, "forward_backward")
        self.dist = dist if dist.is_available() and dist.is_initialized() else None
        self.world = self.dist.get_world_size(group) if self.dist else 1
        if self.world != sampler.W:
            raise ValueError(f"sampler is for {sampler.W} processes, the group has {self.world}")
        self.rank = self.dist.get_rank(group) if self.dist else 0
        buckets = ctx.grad_buckets()
        L = len(buckets) - 2
        # exchange order: the last layer's bucket completes first in the backward
        self.order = list(range(L - 1, -1, -1)) + [L, L + 1]
        self.buckets = buckets
        self.grads = ctx.grads_tensor()
        self.comm = None
        if self.grads.is_cuda:
            import torch
            self.comm = torch.cuda.Stream(device=self.grads.device)

    def exchange(self) -> None:
        """Sum the gradient buckets over the group, each as soon as it is final
        (also in a group of one, whose all-reduce leaves the values as they are)."""
        if self.dist is None:
            return
        if self.comm is None:       # host tensors: the backward has already finished
            for k in self.order:
                o, c = self.buckets[k]
                self.dist.all_reduce(self.grads[o:o + c], group=self.group)
            return
        import torch
        main = torch.cuda.current_stream(self.grads.device)
        with torch.cuda.stream(self.comm):
            for k in self.order:
                self.ctx.grad_wait(k, self.comm)
                o, c = self.buckets[k]
                self.dist.all_reduce(self.grads[o:o + c], group=self.group)
        main.wait_stream(self.comm)

    def step(self, step: int, lr: float, loss_accum=None) -> Shard:
        sh = self.sampler.shard(step)
        b = self.ctx.collate(self.store, sh.ids)
        self.ctx.set_loss_scale(*sh.scales(self.rank))
        if self.captured:
            self.ctx.forward_backward(b, loss_accum)
        else:
            self.ctx.forward(b, train=True)
            self.ctx.backward(b, None, loss_accum)
        self.exchange()
        self.ctx.step(lr)
        return sh
