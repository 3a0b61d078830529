"""torch.autograd.Function wrappers of the library's hand-written gather /
scatter-aggregate and pooling kernels, for composing the PNA layer from
PyTorch (the forward and the backward both run in libgcnn's CUDA kernels).

  Aggregate  PQ (N x 2H, P | Q halves) -> [sum, mean, min, max, std] (N x 5H) of
             m_ij = P_i + Q_j over each destination's CSR row; backward routes
             the gradient to P and to each message's source through the
             reverse-edge slots (min/max ties share equally, std by its chain
             rule), deterministically; given the graph offsets, large batches
             run it fused over chunks of whole graphs.
  MeanPool   node features (N x H) -> per-graph means (G x H); backward spreads
             the gradient evenly over each graph's nodes.
"""
from __future__ import annotations

import torch

from . import aggregate_bwd, aggregate_fwd, pool_bwd, pool_fwd


class Aggregate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, PQ, row_ptr, col, rev, std_eps: float = 1e-5, node_off=None):
        PQ = PQ.contiguous()
        agg = aggregate_fwd(PQ, row_ptr, col, std_eps)
        ctx.save_for_backward(PQ, agg, row_ptr, col, rev)
        ctx.std_eps = std_eps
        ctx.node_off = node_off
        return agg

    @staticmethod
    def backward(ctx, dagg):
        PQ, agg, row_ptr, col, rev = ctx.saved_tensors
        dPQ = aggregate_bwd(PQ, agg, dagg.contiguous(), row_ptr, col, rev, ctx.std_eps, node_off=ctx.node_off)
        return dPQ, None, None, None, None, None


class MeanPool(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, node_off, graph_id):
        x = x.contiguous()
        ctx.save_for_backward(node_off, graph_id)
        ctx.n_nodes = x.shape[0]
        return pool_fwd(x, node_off)

    @staticmethod
    def backward(ctx, dpooled):
        node_off, graph_id = ctx.saved_tensors
        return pool_bwd(dpooled.contiguous(), node_off, graph_id, ctx.n_nodes), None, None


def aggregate(PQ, row_ptr, col, rev, std_eps: float = 1e-5, node_off=None):
    """With the graph offsets node_off (G + 1 int32, no edge leaving its graph) the
    backward runs gcnn_op_aggregate_bwd_graphs (fused over graph chunks on large batches)."""
    return Aggregate.apply(PQ, row_ptr, col, rev, std_eps, node_off)


def mean_pool(x, node_off, graph_id):
    return MeanPool.apply(x, node_off, graph_id)
