"""A second, vectorised statement of the PNA layer in plain PyTorch CPU ops (FP64).

Used only to pin the C oracle: it is written with library routines
(``scatter_reduce`` for sum/mean/min/max, the E[m^2] - E[m]^2 form of the
variance, per-edge messages from ``torch.cat`` + matmul) so that it shares no
structure with the oracle's loops, and its gradients come from autograd.
"""
from __future__ import annotations

import numpy as np
import torch


def _views(d, p):
    H, L, T, Hh = d.H, d.L, d.T, d.Hh
    out, k = {}, 0

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
    if getattr(d, "F", 0):
        k = (k + 3) // 4 * 4          # bond rows start at a multiple of 4 floats
        for l in range(L):
            take(f"edge_w{l}", (d.F, H))
    if getattr(d, "NH", 0):
        k = (k + 3) // 4 * 4          # node head likewise
        take("w1n", (H, Hh))
        take("b1n", (Hh,))
        take("w2n", (Hh,))
        take("b2n", (1,))
    return out


def forward(d, params: torch.Tensor, b, x0: torch.Tensor | None = None, eps: float = 1e-5,
            layers: list | None = None, nodes: list | None = None):
    """Predictions (G,) for a collated batch ``b`` (oracle.Batch) -- autograd-able."""
    W = _views(d, params)
    H = d.H
    N = b.N
    dst = torch.from_numpy(np.repeat(np.arange(N), np.diff(b.row_ptr))).long()
    src = torch.from_numpy(b.col.astype(np.int64))
    deg = torch.from_numpy(b.deg.astype(np.float64))
    has = (deg > 0).double().unsqueeze(1)
    amp = torch.from_numpy(b.amp.astype(np.float64)).unsqueeze(1)
    att = torch.from_numpy(b.att.astype(np.float64)).unsqueeze(1)
    x = W["emb"][torch.from_numpy(b.types.astype(np.int64))] if x0 is None else x0
    if layers is not None:
        layers.append(x)
    idx = dst.unsqueeze(1).expand(-1, H)
    for l in range(d.L):
        mw = W[f"msg_w{l}"]
        WM = torch.cat([mw[:, :H], mw[:, H:]], dim=0)            # (2H, H) acting on [x_i ; x_j]
        inp = [x[dst], x[src]]
        if getattr(d, "F", 0):                                   # bond features: [x_i ; x_j ; e_ij]
            WM = torch.cat([WM, W[f"edge_w{l}"]], dim=0)
            inp.append(torch.from_numpy(b.eattr.astype(np.float64)))
        m = torch.cat(inp, dim=1) @ WM + W[f"msg_b{l}"]
        z = torch.zeros(N, H, dtype=x.dtype)
        s_sum = z.scatter_reduce(0, idx, m, "sum", include_self=False)
        s_mean = z.scatter_reduce(0, idx, m, "mean", include_self=False)
        s_min = z.scatter_reduce(0, idx, m, "amin", include_self=False)
        s_max = z.scatter_reduce(0, idx, m, "amax", include_self=False)
        s_sq = z.scatter_reduce(0, idx, m * m, "mean", include_self=False)
        s_std = torch.sqrt(torch.relu(s_sq - s_mean * s_mean) + eps) * has
        agg = torch.cat([s_sum, s_mean, s_min, s_max, s_std], dim=1) * has
        u = torch.cat([x, agg, agg * amp, agg * att], dim=1)
        x = torch.relu(u @ W[f"upd_w{l}"] + W[f"upd_b{l}"])
        if layers is not None:
            layers.append(x)
    gid = torch.from_numpy(b.graph_id.astype(np.int64))
    cnt = torch.bincount(gid, minlength=b.G).double().clamp(min=1).unsqueeze(1)
    g = torch.zeros(b.G, H, dtype=x.dtype).index_add(0, gid, x) / cnt
    if nodes is not None and getattr(d, "NH", 0):       # node-level head, no pooling
        nodes.append(torch.relu(x @ W["w1n"] + W["b1n"]) @ W["w2n"] + W["b2n"])
    return torch.relu(g @ W["w1"] + W["b1"]) @ W["w2"] + W["b2"]


def loss_and_grads(d, params_np, b, x0_np=None, eps: float = 1e-5):
    p = torch.tensor(params_np, dtype=torch.float64, requires_grad=True)
    x0 = None if x0_np is None else torch.tensor(x0_np, dtype=torch.float64, requires_grad=True)
    nodes = []
    pred = forward(d, p, b, x0, eps, nodes=nodes)
    y = torch.from_numpy(b.y.astype(np.float64))
    loss = torch.mean((pred - y) ** 2)
    if nodes:
        yn = torch.from_numpy(b.ynode.astype(np.float64))
        loss = loss + d.node_weight * torch.mean((nodes[0] - yn) ** 2)
    loss.backward()
    return (float(loss.detach()), p.grad.numpy().copy(), None if x0 is None else x0.grad.numpy().copy(),
            pred.detach().numpy().copy())
