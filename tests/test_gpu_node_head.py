"""Node-level head (Sec. 3.1 node-level properties, Table 1 node-level y): one
output per atom from the last layer, yhat_i = w2n . ReLU(W1n x_i + b1n) + b2n, and
loss = graph MSE + node_weight * node MSE.  The CUDA path against the FP64 oracle:
FP32 forward within 1e-5 (graph and node outputs) and gradients within 1e-4 (every
parameter, the node head included), the captured train step, the recompute path,
BF16 forward within 2e-2 (its gradients within the derived BF16 bound, with the
residual amplification of both losses); a store without node targets is
refused.  FP32 errors are gated normwise and elementwise."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_common import context, oracle_step, write_both
from helpers import FP32_FWD_TOL, FP32_GRAD_TOL, Gates, bf16_grad_bound, rel_norm, residual_kappa

pytestmark = pytest.mark.gpu

W = 0.7


def _workload(G=64, lo=5, hi=30, H=32, L=2, F=0):
    d = oracle.Dims(H=H, L=L, F=F, NH=1, node_weight=W)
    gs = synth.molecules_uniform(61, G, lo, hi)
    gs.y = synth.uniform_targets(62, 0, G, 1.0, 10.0)
    gs.ynode = synth.uniform(63, 0, gs.n_nodes, -1.0, 1.0).astype(np.float32)
    if F:
        gs.eattr = synth.bond_features(64, gs, F, -1.0, 1.0)
    p = synth.init_params(65, H, L, F=F)
    pad = np.zeros((p.size + 3) // 4 * 4 - p.size, np.float32)
    nh = synth.init_params(66, H, 1)[-(H * H + 2 * H + 1):]
    return d, gs, np.concatenate([p, pad, nh])


def _setup(tmp_path, precision=0, recompute=False, resident=True, **kw):
    import paper_2207_11333_gb300 as g
    d, gs, p = _workload(**kw)
    path, ost = write_both(gs, str(tmp_path))
    st = g.Store(path)
    assert st.has_node_targets
    if resident:
        st.to_device()
    delta = st.delta()
    ctx = context(d.H, d.L, gs.n_graphs, gs.n_nodes, gs.n_edges, delta, recompute=recompute, precision=precision,
                  F=d.F, node_head=1, node_weight=W)
    ctx.set_params(p)
    ids = np.arange(gs.n_graphs)
    return d, g, ctx, st, ctx.collate(st, ids), oracle.collate(ost, ids, delta), p


@pytest.mark.parametrize("recompute,resident,F", [(False, True, 0), (True, True, 0), (False, False, 0),
                                                  (False, True, 4)])
def test_fp32_step_with_node_head_matches_oracle(tmp_path, recompute, resident, F):
    d, g, ctx, st, b, ob, p = _setup(tmp_path, recompute=recompute, resident=resident, F=F)
    assert np.array_equal(b.tensor("node_y").cpu().numpy(), ob.ynode)
    pred = torch.empty(b.n_graphs, device="cuda")
    acc = torch.zeros(5, dtype=torch.float64, device="cuda")
    ctx.forward(b, pred, train=True)
    predn = ctx.node_predictions(b)
    ctx.backward(b, None, acc)
    grads = ctx.get_grads()
    ctx.check()
    opred, opredn = oracle.forward(d, p.astype(np.float64), ob, want_nodes=True)
    loss, ograd, _, _ = oracle_step(d, p, ob)
    gates = Gates(f"node head, recompute = {recompute}, F = {F}")
    gates.check("pred", pred.cpu().numpy(), opred, FP32_FWD_TOL)
    gates.check("pred_node", predn, opredn, FP32_FWD_TOL)
    gv, ov = oracle.split_params(d, grads), oracle.split_params(d, ograd)
    for k in ov:
        gates.check(k, gv[k], ov[k], FP32_GRAD_TOL)
    gates.assert_all()
    a = acc.cpu().numpy()
    assert a[2] == b.n_graphs and a[4] == b.n_nodes
    assert abs(a[0] / a[2] + W * a[3] / a[4] - loss) < 1e-5 * loss


def test_captured_train_step_with_node_head(tmp_path):
    d, g, ctx, st, b, ob, p = _setup(tmp_path)
    acc = torch.zeros(5, dtype=torch.float64, device="cuda")
    ctx.train_step(b, 1e-3, acc)
    ctx.check()
    loss, _, _, oth = oracle_step(d, p, ob)
    a = acc.cpu().numpy()
    assert abs(a[0] / a[2] + W * a[3] / a[4] - loss) < 1e-5 * loss
    new = ctx.get_params()
    assert rel_norm(new - p, oth - p) < 1e-3
    assert rel_norm(new, oth) < 1e-5


def test_bf16_with_node_head(tmp_path):
    d, g, ctx, st, b, ob, p = _setup(tmp_path, precision=1)
    pred = torch.empty(b.n_graphs, device="cuda")
    ctx.forward(b, pred, train=True)
    predn = ctx.node_predictions(b)
    ctx.backward(b)
    grads = ctx.get_grads()
    ctx.check()
    opred, opredn = oracle.forward(d, p.astype(np.float64), ob, want_nodes=True)
    _, ograd, _, _ = oracle_step(d, p, ob)
    assert rel_norm(pred.cpu().numpy(), opred) < 2e-2
    assert rel_norm(predn, opredn) < 2e-2
    # the loss gradient is the residual of both heads: the larger amplification
    kappa = max(residual_kappa(opred, ob.y), residual_kappa(opredn, ob.ynode))
    bound = bf16_grad_bound(d.L, kappa)
    gv, ov = oracle.split_params(d, grads), oracle.split_params(d, ograd)
    gates = Gates(f"node head, bf16, bound {bound:.3f}")
    for k in ov:
        gates.check(k, gv[k], ov[k], bound, elementwise=False)
    gates.assert_all()


def test_node_head_needs_node_targets(tmp_path):
    import paper_2207_11333_gb300 as g
    gs = synth.molecules_uniform(67, 8, 5, 12)
    path, _ = write_both(gs, str(tmp_path))
    st = g.Store(path)
    assert not st.has_node_targets
    ctx = context(16, 1, 8, gs.n_nodes, gs.n_edges, st.delta(), node_head=1)
    with pytest.raises(g.GcnnError, match="node targets"):
        ctx.collate(st, np.arange(8))
    srv = g.Server(ctx, n_slots=1, buckets=(1024,), max_graphs=64)   # graph-level screening still serves
    srv.close()


@pytest.mark.parametrize("L,F", [(1, 0), (2, 4)])
def test_bf16_overlapped_train_steps_match_serial(tmp_path, L, F):
    """BF16 train steps with the node head (and bond features): the overlapped
    step, whose AdamW updates of the layers, the head, the bond rows and the node
    head run on a third stream during the backward, equals the serial step (one
    update at the end) bit for bit, parameters and loss sums; L = 1 has no
    per-layer early update, only layer 0's beside the embedding gradient."""
    import paper_2207_11333_gb300 as g
    d, gs, p = _workload(G=96, lo=3, hi=40, H=32, L=L, F=F)
    path, _ = write_both(gs, str(tmp_path))
    st = g.Store(path)
    delta = st.delta()
    res = []
    for flags in (0, g.FLAG_SERIAL):
        ctx = g.Context(g.make_config(d.H, L, gs.n_graphs, gs.n_nodes, gs.n_edges, delta=delta,
                                      precision=g.PREC_BF16, flags=flags, head_hidden=d.H, edge_features=F,
                                      node_head=1, node_loss_weight=W))
        ctx.set_params(p)
        acc = torch.zeros(5, dtype=torch.float64, device="cuda")
        for k in range(3):
            ids = np.random.default_rng(k).permutation(gs.n_graphs)
            ctx.train_step(ctx.collate(st, ids), 1e-3, acc)
        res.append((ctx.get_params(), acc.cpu().numpy()))
        ctx.check()
        ctx.close()
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1], res[1][1])
