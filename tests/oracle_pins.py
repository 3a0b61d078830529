"""Pins of the FP64 oracle against facts fixed outside it.

Each ``pin_*`` function raises AssertionError when the oracle disagrees with an
independent statement: a textbook identity, a library routine, a closed form,
an invariance, or finite differences.  The same functions run against
deliberately broken copies of the oracle in test_oracle_mutations.py, which
checks that each planted mistake is caught by at least one pin.
"""
from __future__ import annotations

import math

import numpy as np
import torch

import oracle
import synth
import torch_ref
from helpers import custom_set, graph_set, oracle_batch, rel_max, rel_norm, star_and_dense_set

EPS = 1e-5


def _model(seed: int, H: int, L: int):
    d = oracle.Dims(H=H, L=L)
    p = synth.init_params(seed, H, L).astype(np.float64)
    return d, p


def pin_collation_lexsort():
    """Row order equals numpy lexsort by (dst, src); reverse edges are consistent."""
    gs = graph_set(1, 24, 3, 30)
    ids = synth.node_counts_uniform(5, 0, 24, 1, 24).astype(np.int64) - 1   # shuffled order, repeats allowed
    st, b, _ = oracle_batch(gs, ids)
    src, dst = [], []
    off = 0
    for g in ids:
        e = gs.edges[gs.edge_ptr[g]:gs.edge_ptr[g + 1]].astype(np.int64)
        src.append(e[:, 0] + off)
        dst.append(e[:, 1] + off)
        off += gs.node_ptr[g + 1] - gs.node_ptr[g]
    src, dst = np.concatenate(src), np.concatenate(dst)
    order = np.lexsort((src, dst))
    assert np.array_equal(b.col, src[order].astype(np.int32))
    rp = np.zeros(b.N + 1, np.int64)
    rp[1:] = np.cumsum(np.bincount(dst, minlength=b.N))
    assert np.array_equal(b.row_ptr, rp.astype(np.int32))
    assert np.array_equal(b.deg, np.diff(rp).astype(np.int32))
    d_of_e = dst[order]
    assert np.array_equal(b.rev[b.rev], np.arange(b.E))
    assert np.array_equal(b.col[b.rev], d_of_e.astype(np.int32))
    n = gs.node_ptr[ids + 1] - gs.node_ptr[ids]
    assert np.array_equal(b.graph_id, np.repeat(np.arange(len(ids)), n).astype(np.int32))
    assert np.array_equal(b.types, np.concatenate([gs.types[gs.node_ptr[g]:gs.node_ptr[g + 1]] for g in ids]))
    assert np.array_equal(b.y, gs.y[ids])


def pin_sum_is_dense_adjacency_matmul():
    """sum_j m_ij = d_i (x_i A + b) + sum_j x_j B  =  (D X A + d b^T) + Adj X B  (dense matmul)."""
    d, p = _model(3, 8, 2)
    gs = graph_set(1, 6, 5, 14)
    st, b, _ = oracle_batch(gs)
    x0 = synth.normal(21, 0, b.N * d.H).reshape(b.N, d.H)
    pred, xs, ag, _ = oracle.forward(d, p, b, x0=x0, want_layers=True)
    W = oracle.split_params(d, p)
    adj = np.zeros((b.N, b.N))
    for i in range(b.N):
        for e in range(b.row_ptr[i], b.row_ptr[i + 1]):
            adj[i, b.col[e]] += 1.0
    for l in range(d.L):
        x = xs[l]
        A, B = W[f"msg_w{l}"][:, :d.H], W[f"msg_w{l}"][:, d.H:]
        deg = adj.sum(1, keepdims=True)
        expect = deg * (x @ A + W[f"msg_b{l}"]) + adj @ (x @ B)
        assert rel_norm(ag[l][:, :d.H], expect) < 1e-13


def pin_aggregators_scatter_reduce():
    """All five aggregators and each layer's output against torch scatter_reduce + matmul."""
    d, p = _model(3, 16, 3)
    gs = graph_set(2, 10, 5, 20)
    st, b, _ = oracle_batch(gs)
    pred, xs, ag, _ = oracle.forward(d, p, b, want_layers=True)
    layers = []
    ref = torch_ref.forward(d, torch.tensor(p), b, layers=layers).numpy()
    for l in range(d.L + 1):
        assert rel_norm(xs[l], layers[l].numpy()) < 1e-12, l
    assert rel_norm(pred, ref) < 1e-12


def pin_scalers_cycle_closed_form():
    """On cycles every degree is 2: delta = log 3, amplification = attenuation = 1."""
    gs = custom_set([([1] * n, [(k, (k + 1) % n) for k in range(n)]) for n in (3, 5, 8)])
    st, b, delta = oracle_batch(gs)
    assert abs(delta - math.log(3.0)) < 1e-15
    assert np.all(b.amp == np.float32(1.0)) and np.all(b.att == np.float32(1.0))
    assert np.all(b.deg == 2)


def pin_scalers_star_closed_form():
    """Star K_{1,k}: delta = (log(k+1) + k log 2)/(k+1); amp_centre = log(k+1)/delta."""
    for k in (1, 3, 4, 7):
        gs = custom_set([([1] + [0] * k, [(0, j) for j in range(1, k + 1)])])
        st, b, delta = oracle_batch(gs)
        want = (math.log(k + 1) + k * math.log(2.0)) / (k + 1)
        assert abs(delta - want) < 1e-15 * max(1.0, want)
        assert b.amp[0] == np.float32(math.log(k + 1) / want)
        assert b.att[0] == np.float32(want / math.log(k + 1))
        assert np.all(b.amp[1:] == np.float32(math.log(2.0) / want))


def pin_permutation_invariance():
    """Relabelling nodes inside graphs and reordering graphs permutes the predictions only."""
    d, p = _model(3, 12, 2)
    gs = graph_set(4, 12, 5, 25)
    st, b, delta = oracle_batch(gs)
    pred = oracle.forward(d, p, b)
    rng = np.random.default_rng(0)
    graphs = []
    for g in range(gs.n_graphs):
        n = int(gs.node_ptr[g + 1] - gs.node_ptr[g])
        perm = rng.permutation(n)               # new label of old node v is perm[v]
        t = np.empty(n, np.uint8)
        t[perm] = gs.types[gs.node_ptr[g]:gs.node_ptr[g + 1]]
        e = gs.edges[gs.edge_ptr[g]:gs.edge_ptr[g + 1]].astype(np.int64)
        und = [(perm[u], perm[v]) for u, v in e[::2]]
        graphs.append((t.tolist(), und))
    gs2 = custom_set(graphs)
    gs2.y = gs.y.copy()
    order = rng.permutation(gs.n_graphs)
    st2, b2, delta2 = oracle_batch(gs2, order)
    assert abs(delta2 - delta) < 1e-14
    pred2 = oracle.forward(d, p, b2)
    assert rel_norm(pred2, pred[order]) < 1e-12


def pin_pool_of_constant_graph():
    """A regular graph whose nodes all carry the same input pools to that node's value."""
    d, p = _model(5, 8, 2)
    gs = custom_set([([2] * 6, [(k, (k + 1) % 6) for k in range(6)])])
    st, b, _ = oracle_batch(gs)
    x0 = np.tile(synth.normal(7, 0, d.H), (b.N, 1))
    pred, xs, ag, pooled = oracle.forward(d, p, b, x0=x0, want_layers=True)
    assert np.allclose(xs[d.L], xs[d.L][0:1], rtol=0, atol=1e-14)
    assert rel_norm(pooled[0], xs[d.L][0]) < 1e-14


def pin_constant_messages():
    """Identical messages: min = max = mean = sum/d and std = sqrt(eps)."""
    d, p = _model(6, 8, 1)
    gs = custom_set([([3] * 5, [(k, (k + 1) % 5) for k in range(5)])])
    st, b, _ = oracle_batch(gs)
    x0 = np.tile(synth.normal(8, 0, d.H), (b.N, 1))
    _, xs, ag, _ = oracle.forward(d, p, b, x0=x0, want_layers=True)
    H = d.H
    a = ag[0]
    assert np.allclose(a[:, 2 * H:3 * H], a[:, H:2 * H], rtol=1e-15, atol=0)
    assert np.allclose(a[:, 3 * H:4 * H], a[:, H:2 * H], rtol=1e-15, atol=0)
    assert np.allclose(a[:, 0:H], 2 * a[:, H:2 * H], rtol=1e-15, atol=0)
    assert np.allclose(a[:, 4 * H:5 * H], math.sqrt(EPS), rtol=1e-15, atol=0)


def pin_gradients_autograd():
    """Hand-written gradients equal torch autograd (FP64), with atom-type embeddings (min/max ties)."""
    d, p = _model(3, 12, 2)
    gs = graph_set(1, 8, 5, 16)
    st, b, _ = oracle_batch(gs)
    loss, grad, _, pred = oracle.backward(d, p, b)
    rloss, rgrad, _, rpred = torch_ref.loss_and_grads(d, p, b)
    assert abs(loss - rloss) <= 1e-12 * abs(rloss)
    assert rel_norm(pred, rpred) < 1e-12
    views, rviews = oracle.split_params(d, grad), oracle.split_params(d, rgrad)
    for k in views:
        assert rel_norm(views[k], rviews[k]) < 1e-10, k


def pin_gradients_autograd_continuous():
    """Gradients w.r.t. parameters and node inputs equal torch autograd with continuous inputs."""
    d, p = _model(4, 8, 3)
    gs = graph_set(20, 6, 5, 12)
    st, b, _ = oracle_batch(gs)
    x0 = synth.normal(22, 0, b.N * d.H).reshape(b.N, d.H)
    loss, grad, dx0, _ = oracle.backward(d, p, b, x0=x0)
    rloss, rgrad, rdx0, _ = torch_ref.loss_and_grads(d, p, b, x0)
    assert abs(loss - rloss) <= 1e-12 * abs(rloss)
    views, rviews = oracle.split_params(d, grad), oracle.split_params(d, rgrad)
    for k in views:
        if k == "emb":
            continue
        assert rel_norm(views[k], rviews[k]) < 1e-10, k
    assert rel_norm(dx0, rdx0) < 1e-10


def pin_finite_differences(n_coords: int = 400):
    """Central differences (h = 1e-6, FP64) of the MSE loss against the analytic gradient,
    on 16 graphs of 5-12 nodes with continuous node inputs (no min/max ties)."""
    d, p = _model(3, 8, 2)
    gs = graph_set(20, 16, 5, 12)
    st, b, _ = oracle_batch(gs)
    x0 = synth.normal(23, 0, b.N * d.H).reshape(b.N, d.H)
    loss0, grad, dx0, _ = oracle.backward(d, p, b, x0=x0)
    h = 1e-6
    rng = np.random.default_rng(1)
    emb = d.T * d.H
    coords = rng.choice(np.arange(emb, p.size), size=min(n_coords, p.size - emb), replace=False)
    fd = np.empty(len(coords))
    for n, k in enumerate(coords):
        q = p.copy()
        q[k] += h
        lp = oracle.backward(d, q, b, x0=x0)[0]
        q[k] -= 2 * h
        lm = oracle.backward(d, q, b, x0=x0)[0]
        fd[n] = (lp - lm) / (2 * h)
    an = grad[coords]
    # central differences carry O(h^2) truncation plus a rounding floor of about
    # eps_mach * |L| / h; allow 1e-6 relative on top of 20x that floor
    floor = 20 * np.finfo(np.float64).eps * abs(loss0) / h
    bad = np.abs(fd - an) > 1e-6 * np.abs(an) + floor
    assert not bad.any(), (bad.sum(), coords[bad][:5])
    assert rel_norm(fd, an) < 1e-6
    # node inputs
    ids = rng.choice(b.N * d.H, size=60, replace=False)
    fdx = np.empty(len(ids))
    for n, k in enumerate(ids):
        y = x0.copy().ravel()
        y[k] += h
        lp = oracle.backward(d, p, b, x0=y.reshape(x0.shape))[0]
        y[k] -= 2 * h
        lm = oracle.backward(d, p, b, x0=y.reshape(x0.shape))[0]
        fdx[n] = (lp - lm) / (2 * h)
    assert np.all(np.abs(fdx - dx0.ravel()[ids]) <= 1e-6 * np.abs(dx0.ravel()[ids]) + floor)


def pin_adam_first_step():
    """First Adam step: theta1 = theta0 - lr * g / (|g| + eps) (bias corrections cancel)."""
    rng = np.random.default_rng(2)
    th = rng.standard_normal(1000)
    g = rng.standard_normal(1000) * np.exp(rng.uniform(-8, 2, 1000))
    m, v = np.zeros(1000), np.zeros(1000)
    t0 = th.copy()
    oracle.adam(th, g, m, v, 1, lr=1e-3)
    assert rel_max(th - t0, -1e-3 * g / (np.abs(g) + 1e-8)) < 1e-9
    # second step with zero gradient: m1 = 0.1 g -> m2 = 0.09 g ; v2 = 0.999 * 0.001 g^2
    t1 = th.copy()
    oracle.adam(th, np.zeros(1000), m, v, 2, lr=1e-3)
    mh = 0.09 * g / (1 - 0.9 ** 2)
    vh = 0.999 * 0.001 * g * g / (1 - 0.999 ** 2)
    assert rel_max(th - t1, -1e-3 * mh / (np.sqrt(vh) + 1e-8)) < 1e-9


def pin_adamw_decay():
    """Zero gradient, first step: AdamW only shrinks theta by lr * wd * theta."""
    th = np.linspace(-2, 2, 64)
    t0 = th.copy()
    oracle.adam(th, np.zeros(64), np.zeros(64), np.zeros(64), 1, lr=1e-2, wd=0.1)
    assert rel_max(th, t0 * (1 - 1e-3)) < 1e-15


def pin_mse_gradient():
    """dL/dpred = 2 (pred - y) / G: the backward with an explicit dpred equals the MSE path."""
    d, p = _model(3, 8, 2)
    gs = graph_set(6, 7, 5, 15)
    st, b, _ = oracle_batch(gs)
    loss, grad, _, pred = oracle.backward(d, p, b)
    assert abs(loss - float(np.mean((pred - b.y.astype(np.float64)) ** 2))) < 1e-13 * loss
    _, grad2, _, _ = oracle.backward(d, p, b, dpred=2.0 * (pred - b.y) / b.G)
    assert rel_norm(grad2, grad) < 1e-14


def _bond_model(seed: int, H: int, L: int, F: int):
    d = oracle.Dims(H=H, L=L, F=F)
    p = synth.init_params(seed, H, L, F=F).astype(np.float64)
    return d, p


def _with_bonds(gs, F, seed=31):
    gs.eattr = synth.bond_features(seed, gs, F, -1.0, 1.0)
    return gs


def pin_bond_features_collated_with_their_edge():
    """Each collated edge carries the features stored for that (source, destination) pair."""
    gs = _with_bonds(graph_set(7, 10, 3, 30), 3)
    ids = np.array([4, 1, 9, 1, 0], np.int64)
    st, b, _ = oracle_batch(gs, ids)
    stored = {}
    off = 0
    for g in ids:
        e0, e1 = gs.edge_ptr[g], gs.edge_ptr[g + 1]
        for k in range(e0, e1):
            s_, t_ = (int(v) + off for v in gs.edges[k])
            stored[(s_, t_)] = gs.eattr[k]
        off += int(gs.node_ptr[g + 1] - gs.node_ptr[g])
    dst = np.repeat(np.arange(b.N), np.diff(b.row_ptr))
    for p_ in range(b.E):
        assert np.array_equal(b.eattr[p_], stored[(int(b.col[p_]), int(dst[p_]))])


def pin_bond_features_zero_weights():
    """Zero bond rows: the model with bond features equals the model without them."""
    d, p = _bond_model(3, 8, 2, 4)
    d0, p0 = _model(3, 8, 2)
    assert np.array_equal(p[:p0.size], p0)
    q = p.copy()
    q[p0.size:] = 0.0
    gs = graph_set(8, 9, 5, 20)
    gs.y = synth.uniform_targets(9, 0, gs.n_graphs, 1, 10)
    _, b0, _ = oracle_batch(gs)
    _, b, _ = oracle_batch(_with_bonds(gs, 4))
    assert np.array_equal(oracle.forward(d, q, b), oracle.forward(d0, p0, b0))
    l, g, _, _ = oracle.backward(d, q, b)
    l0, g0, _, _ = oracle.backward(d0, p0, b0)
    assert l == l0 and np.array_equal(g[:p0.size], g0)


def pin_bond_features_constant_is_bias_shift():
    """Every bond carrying the same features v is a shift of the message bias by v W_E."""
    d, p = _bond_model(4, 8, 2, 3)
    d0 = oracle.Dims(H=8, L=2)
    gs = graph_set(10, 8, 5, 16)
    v = np.array([0.5, -1.25, 2.0], np.float32)
    gs.eattr = np.tile(v, (gs.n_edges, 1))
    _, b, _ = oracle_batch(gs)
    gs0 = graph_set(10, 8, 5, 16)
    _, b0, _ = oracle_batch(gs0)
    W = oracle.split_params(d, p)
    q = p[:oracle.param_count(d0)].copy()
    V = oracle.split_params(d0, q)
    for l in range(d.L):
        V[f"msg_b{l}"][:] += v.astype(np.float64) @ W[f"edge_w{l}"]
    assert rel_norm(oracle.forward(d, p, b), oracle.forward(d0, q, b0)) < 1e-12


def pin_bond_features_autograd():
    """With bond features, gradients (bond rows included) equal torch autograd (FP64)."""
    d, p = _bond_model(5, 8, 2, 4)
    gs = _with_bonds(graph_set(21, 6, 5, 12), 4)
    gs.y = synth.uniform_targets(22, 0, gs.n_graphs, 1, 10)
    _, b, _ = oracle_batch(gs)
    x0 = synth.normal(24, 0, b.N * d.H).reshape(b.N, d.H)
    loss, grad, dx0, _ = oracle.backward(d, p, b, x0=x0)
    rloss, rgrad, rdx0, _ = torch_ref.loss_and_grads(d, p, b, x0)
    assert abs(loss - rloss) <= 1e-12 * abs(rloss)
    views, rviews = oracle.split_params(d, grad), oracle.split_params(d, rgrad)
    for k in views:
        if k != "emb":
            assert rel_norm(views[k], rviews[k]) < 1e-10, k
    assert rel_norm(dx0, rdx0) < 1e-10


def pin_bond_features_finite_differences():
    """Central differences of the loss w.r.t. the bond rows and the message weights."""
    d, p = _bond_model(6, 6, 2, 3)
    gs = _with_bonds(graph_set(25, 8, 5, 12), 3)
    gs.y = synth.uniform_targets(26, 0, gs.n_graphs, 1, 10)
    _, b, _ = oracle_batch(gs)
    x0 = synth.normal(27, 0, b.N * d.H).reshape(b.N, d.H)
    loss0, grad, _, _ = oracle.backward(d, p, b, x0=x0)
    base = oracle.param_count(oracle.Dims(H=d.H, L=d.L))
    coords = np.concatenate([np.arange(base, p.size), np.arange(d.T * d.H, d.T * d.H + 40)])
    h = 1e-6
    fd = np.empty(len(coords))
    for n, k in enumerate(coords):
        q = p.copy()
        q[k] += h
        lp = oracle.backward(d, q, b, x0=x0)[0]
        q[k] -= 2 * h
        lm = oracle.backward(d, q, b, x0=x0)[0]
        fd[n] = (lp - lm) / (2 * h)
    floor = 20 * np.finfo(np.float64).eps * abs(loss0) / h
    assert np.all(np.abs(fd - grad[coords]) <= 1e-6 * np.abs(grad[coords]) + floor)


def pin_bond_features_permutation_invariance():
    """Relabelling nodes (bond features travel with their bonds) and reordering graphs."""
    d, p = _bond_model(7, 8, 2, 2)
    gs = _with_bonds(graph_set(28, 10, 5, 20), 2)
    _, b, _ = oracle_batch(gs)
    pred = oracle.forward(d, p, b)
    rng = np.random.default_rng(3)
    graphs, attrs = [], []
    for g in range(gs.n_graphs):
        n = int(gs.node_ptr[g + 1] - gs.node_ptr[g])
        perm = rng.permutation(n)
        t = np.empty(n, np.uint8)
        t[perm] = gs.types[gs.node_ptr[g]:gs.node_ptr[g + 1]]
        e = gs.edges[gs.edge_ptr[g]:gs.edge_ptr[g + 1]].astype(np.int64)
        a = gs.eattr[gs.edge_ptr[g]:gs.edge_ptr[g + 1]]
        bonds = rng.permutation(len(e) // 2)
        graphs.append((t.tolist(), [(perm[e[2 * k, 0]], perm[e[2 * k, 1]]) for k in bonds]))
        attrs.append(np.repeat(a[2 * bonds], 2, axis=0))
    gs2 = custom_set(graphs)
    gs2.eattr = np.ascontiguousarray(np.concatenate(attrs))
    order = rng.permutation(gs.n_graphs)
    _, b2, _ = oracle_batch(gs2, order)
    assert rel_norm(oracle.forward(d, p, b2), pred[order]) < 1e-12


def _node_model(seed: int, H: int, L: int, weight: float = 1.0):
    d = oracle.Dims(H=H, L=L, NH=1, node_weight=weight)
    base = synth.init_params(seed, H, L).astype(np.float64)
    head = synth.init_params(seed + 100, H, 1).astype(np.float64)    # reuse a head block's draws
    hs = H * H + 2 * H + 1
    pad = np.zeros((base.size + 3) // 4 * 4 - base.size)
    return d, np.concatenate([base, pad, head[-hs:]])


def _with_node_targets(gs, seed=51):
    gs.ynode = synth.uniform(seed, 0, gs.n_nodes, -1.0, 1.0).astype(np.float32)
    return gs


def pin_node_head_weight_zero():
    """Node-loss weight 0: the trunk and graph-head gradients equal those of the model
    without a node head, and the node head's own gradients vanish."""
    d, p = _node_model(3, 8, 2, weight=0.0)
    d0 = oracle.Dims(H=8, L=2)
    n0 = oracle.param_count(d0)
    gs = _with_node_targets(graph_set(9, 8, 5, 18))
    _, b, _ = oracle_batch(gs)
    l, g, _, _ = oracle.backward(d, p, b)
    l0, g0, _, _ = oracle.backward(d0, p[:n0], b)
    assert l == l0 and np.array_equal(g[:n0], g0) and not np.any(g[n0:])


def pin_node_head_constant_output():
    """W1n = 0: every atom predicts c = w2n . ReLU(b1n) + b2n, the node loss is
    mean((c - y_i)^2) and its gradient w.r.t. b2n is weight * 2 mean(c - y_i)."""
    d, p = _node_model(4, 8, 1, weight=0.75)
    V = oracle.split_params(d, p)
    V["w1n"][:] = 0.0
    gs = _with_node_targets(graph_set(11, 7, 5, 15))
    _, b, _ = oracle_batch(gs)
    pred, predn = oracle.forward(d, p, b, want_nodes=True)
    c = float(np.maximum(V["b1n"], 0.0) @ V["w2n"] + V["b2n"][0])
    assert np.allclose(predn, c, rtol=0, atol=1e-14)
    loss, grad, _, _ = oracle.backward(d, p, b)
    yn = b.ynode.astype(np.float64)
    graph_mse = np.mean((pred - b.y.astype(np.float64)) ** 2)
    assert abs(loss - (graph_mse + 0.75 * np.mean((c - yn) ** 2))) < 1e-12 * loss
    G = oracle.split_params(d, grad)
    assert abs(G["b2n"][0] - 0.75 * 2.0 * np.mean(c - yn)) < 1e-12


def pin_node_head_autograd():
    """With a node head, every gradient equals torch autograd (FP64)."""
    d, p = _node_model(5, 8, 2, weight=0.5)
    gs = _with_node_targets(graph_set(23, 6, 5, 12))
    gs.y = synth.uniform_targets(24, 0, gs.n_graphs, 1, 10)
    _, b, _ = oracle_batch(gs)
    x0 = synth.normal(25, 0, b.N * d.H).reshape(b.N, d.H)
    loss, grad, dx0, _ = oracle.backward(d, p, b, x0=x0)
    rloss, rgrad, rdx0, _ = torch_ref.loss_and_grads(d, p, b, x0)
    assert abs(loss - rloss) <= 1e-12 * abs(rloss)
    views, rviews = oracle.split_params(d, grad), oracle.split_params(d, rgrad)
    for k in views:
        if k != "emb":
            assert rel_norm(views[k], rviews[k]) < 1e-10, k
    assert rel_norm(dx0, rdx0) < 1e-10


def pin_node_head_finite_differences():
    """Central differences of the multitask loss w.r.t. the node head and the last layer."""
    d, p = _node_model(6, 6, 1, weight=1.3)
    gs = _with_node_targets(graph_set(26, 8, 5, 12))
    gs.y = synth.uniform_targets(27, 0, gs.n_graphs, 1, 10)
    _, b, _ = oracle_batch(gs)
    x0 = synth.normal(28, 0, b.N * d.H).reshape(b.N, d.H)
    loss0, grad, _, _ = oracle.backward(d, p, b, x0=x0)
    n0 = oracle.param_count(oracle.Dims(H=d.H, L=d.L))
    coords = np.concatenate([np.arange((n0 + 3) // 4 * 4, p.size), np.arange(d.T * d.H, d.T * d.H + 40)])
    h = 1e-6
    fd = np.empty(len(coords))
    for n, k in enumerate(coords):
        q = p.copy()
        q[k] += h
        lp = oracle.backward(d, q, b, x0=x0)[0]
        q[k] -= 2 * h
        lm = oracle.backward(d, q, b, x0=x0)[0]
        fd[n] = (lp - lm) / (2 * h)
    floor = 20 * np.finfo(np.float64).eps * abs(loss0) / h
    assert np.all(np.abs(fd - grad[coords]) <= 1e-6 * np.abs(grad[coords]) + floor)


def pin_node_head_permutation_equivariance():
    """Relabelling atoms permutes the node-level predictions the same way."""
    d, p = _node_model(7, 8, 2)
    gs = graph_set(29, 6, 5, 14)
    _, b, _ = oracle_batch(gs)
    _, predn = oracle.forward(d, p, b, want_nodes=True)
    rng = np.random.default_rng(4)
    graphs, perms = [], []
    for g in range(gs.n_graphs):
        n = int(gs.node_ptr[g + 1] - gs.node_ptr[g])
        perm = rng.permutation(n)
        t = np.empty(n, np.uint8)
        t[perm] = gs.types[gs.node_ptr[g]:gs.node_ptr[g + 1]]
        e = gs.edges[gs.edge_ptr[g]:gs.edge_ptr[g + 1]].astype(np.int64)
        graphs.append((t.tolist(), [(perm[u], perm[v]) for u, v in e[::2]]))
        perms.append(perm + int(gs.node_ptr[g]))
    _, b2, _ = oracle_batch(custom_set(graphs))
    _, predn2 = oracle.forward(d, p, b2, want_nodes=True)
    assert rel_norm(predn2[np.concatenate(perms)], predn) < 1e-12


def _torch_aggregators(m, row_ptr, eps=EPS):
    """[sum, mean, min, max, std] of per-slot messages by scatter_reduce (FP64, autograd-able)."""
    N = len(row_ptr) - 1
    deg = np.diff(row_ptr)
    dst = torch.from_numpy(np.repeat(np.arange(N), deg)).long()
    idx = dst.unsqueeze(1).expand(-1, m.shape[1])
    z = torch.zeros(N, m.shape[1], dtype=m.dtype)
    s = z.scatter_reduce(0, idx, m, "sum", include_self=False)
    mean = z.scatter_reduce(0, idx, m, "mean", include_self=False)
    mn = z.scatter_reduce(0, idx, m, "amin", include_self=False)
    mx = z.scatter_reduce(0, idx, m, "amax", include_self=False)
    d = torch.from_numpy(np.maximum(deg, 1).astype(np.float64)).unsqueeze(1)
    var = z.index_add(0, dst, m * m) / d - mean * mean       # E[m^2] - E[m]^2
    sd = torch.sqrt(torch.relu(var) + eps)
    has = torch.from_numpy((deg > 0).astype(np.float64)).unsqueeze(1)
    return torch.cat([s, mean, mn, mx, sd], 1) * has


def pin_aggregate_operator_high_degree():
    """The aggregation operator and its per-edge backward against torch
    scatter_reduce + autograd on stars K_{1,k} (k up to 254) and molecules with
    degrees up to 16: continuous messages, and messages on a grid of 1/16 where
    min/max tie among many edges (autograd of amax/amin shares the gradient
    equally among ties, the rule the oracle states).  On the grid P is an odd
    and Q an even multiple of 1/16, so no message is 0: torch's amax/amin
    backward would count the 0 it starts from as one more tie."""
    gs = star_and_dense_set()
    _, b, _ = oracle_batch(gs)
    assert b.deg.max() == 254 and np.sum(b.deg > 4) > 20
    H = 6
    rng = np.random.default_rng(3)
    dst = np.repeat(np.arange(b.N), b.deg)
    for grid in (False, True):
        if grid:   # m_e = P_i + Q_j, odd multiples of 1/16: exact, with ties, never 0
            P, Q = (2 * rng.integers(-8, 8, (b.N, H)) + 1) / 16.0, 2 * rng.integers(-3, 3, (b.N, H)) / 16.0
        else:
            P, Q = rng.standard_normal((b.N, H)), rng.standard_normal((b.N, H))
        m = P[dst] + Q[b.col]
        agg = oracle.aggregate_op(b.row_ptr, m)
        mt = torch.tensor(m, requires_grad=True)
        ref = _torch_aggregators(mt, b.row_ptr)
        assert rel_norm(agg, ref.detach().numpy()) < 1e-12
        assert rel_max(agg, ref.detach().numpy()) < 1e-10
        dagg = rng.standard_normal((b.N, 5 * H))
        (ref * torch.tensor(dagg)).sum().backward()
        dm = oracle.aggregate_bwd_op(b.row_ptr, m, agg, dagg)
        assert rel_norm(dm, mt.grad.numpy()) < 1e-10, grid
        assert rel_max(dm, mt.grad.numpy()) < 1e-8, grid


def pin_gradients_autograd_high_degree():
    """Model gradients equal torch autograd (FP64) on stars and high-degree molecules
    (rows longer than any fixed cache of edges), with atom-type embeddings (ties)."""
    d, p = _model(3, 8, 2)
    gs = star_and_dense_set(ks=(5, 9, 17, 40), dense=4)
    gs.y = synth.uniform_targets(5, 0, gs.n_graphs, 1.0, 10.0)
    st, b, _ = oracle_batch(gs)
    assert b.deg.max() == 40
    loss, grad, _, pred = oracle.backward(d, p, b)
    rloss, rgrad, _, rpred = torch_ref.loss_and_grads(d, p, b)
    assert abs(loss - rloss) <= 1e-12 * abs(rloss)
    assert rel_norm(pred, rpred) < 1e-12
    views, rviews = oracle.split_params(d, grad), oracle.split_params(d, rgrad)
    for k in views:
        assert rel_norm(views[k], rviews[k]) < 1e-10, k


NODE_PINS = [pin_node_head_weight_zero, pin_node_head_constant_output, pin_node_head_autograd,
             pin_node_head_finite_differences, pin_node_head_permutation_equivariance]

BOND_PINS = [pin_bond_features_collated_with_their_edge, pin_bond_features_zero_weights,
             pin_bond_features_constant_is_bias_shift, pin_bond_features_autograd,
             pin_bond_features_finite_differences, pin_bond_features_permutation_invariance]

ALL_PINS = [pin_collation_lexsort, pin_sum_is_dense_adjacency_matmul, pin_aggregators_scatter_reduce,
            pin_scalers_cycle_closed_form, pin_scalers_star_closed_form, pin_permutation_invariance,
            pin_pool_of_constant_graph, pin_constant_messages, pin_gradients_autograd,
            pin_gradients_autograd_continuous, pin_finite_differences, pin_adam_first_step,
            pin_adamw_decay, pin_mse_gradient, pin_aggregate_operator_high_degree,
            pin_gradients_autograd_high_degree] + BOND_PINS + NODE_PINS
