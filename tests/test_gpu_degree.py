"""Rows longer than the aggregation kernels' register cache of four edges,
against the FP64 oracle (Sec. 3.1: sum, mean, min, max and std over every
neighbour).

The batches hold stars K_{1,k} (k = 5, 8, 16, 64, 254: the centre's row has k
edges, its leaves cycle over the atom types, so min/max tie among many edges)
and molecule-shaped graphs with up to 16 bonds per atom.  The large batches
have more than 2 x 152 x 128 edges, so the backward runs fused over chunks of
whole graphs, and the 254-leaf star has more edges (508) than a chunk keeps in
shared memory (192), so its chunk takes the device-memory branch.

Operators: gcnn_op_aggregate_fwd / _bwd / _bwd_graphs against
oracle_aggregate_op / _bwd_op on the same FP32 inputs, on a grid of 1/16 where
every message is exact and ties are decided identically, and on continuous
values.  Model: forward, every layer and every gradient of the FP32 path
(1e-5 / 1e-4, normwise and elementwise), and of the BF16 path (forward 2e-2,
gradients within the derived BF16 bound), with and without bond features.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_common import context, write_both
from helpers import (BF16_FWD_TOL, FP32_FWD_TOL, FP32_GRAD_TOL, Gates, bf16_grad_bound, oracle_batch,
                     residual_kappa, star_and_dense_set)

pytestmark = pytest.mark.gpu

STARS = (5, 8, 16, 64, 254)


def _set(big: bool, seed: int = 51):
    if big:
        return star_and_dense_set(seed=seed, ks=STARS * 40, dense=300)
    return star_and_dense_set(seed=seed, ks=STARS, dense=24)


@pytest.mark.parametrize("grid", [True, False], ids=["grid", "continuous"])
@pytest.mark.parametrize("big", [False, True], ids=["pair", "fused"])
def test_aggregate_operators_high_degree_vs_oracle(big, grid):
    import paper_2207_11333_gb300 as g
    gs = _set(big)
    _, b, _ = oracle_batch(gs)
    assert b.deg.max() == 254 and np.sum(b.deg > 4) > 50
    if big:
        assert b.E > 2 * 152 * 128
    H = 8 if big else 12
    rng = np.random.default_rng(7 + big)
    if grid:   # P odd, Q even multiples of 1/16: every message and every sum is exact in FP32
        P = (2 * rng.integers(-8, 8, (b.N, H)) + 1) / 16.0
        Q = 2 * rng.integers(-3, 3, (b.N, H)) / 16.0
    else:
        P, Q = rng.standard_normal((b.N, H)), rng.standard_normal((b.N, H))
    PQ32 = np.concatenate([P, Q], 1).astype(np.float32)
    dagg32 = rng.standard_normal((b.N, 5 * H)).astype(np.float32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rp, col, rev, no = dev(b.row_ptr), dev(b.col), dev(b.rev), dev(b.node_off.astype(np.int32))
    PQ, dagg = dev(PQ32), dev(dagg32)
    agg = g.aggregate_fwd(PQ, rp, col)
    pair = g.aggregate_bwd(PQ, agg, dagg, rp, col, rev)
    fused = g.aggregate_bwd(PQ, agg, dagg, rp, col, rev, node_off=no)
    torch.cuda.synchronize()
    assert torch.equal(pair, fused)

    P64, Q64 = PQ32[:, :H].astype(np.float64), PQ32[:, H:].astype(np.float64)
    dst = np.repeat(np.arange(b.N), b.deg)
    m = P64[dst] + Q64[b.col]
    oagg = oracle.aggregate_op(b.row_ptr, m)
    odm = oracle.aggregate_bwd_op(b.row_ptr, m, oagg, dagg32.astype(np.float64))
    odP, odQ = np.zeros((b.N, H)), np.zeros((b.N, H))
    np.add.at(odP, dst, odm)
    np.add.at(odQ, b.col, odm)
    gates = Gates(f"aggregation operators, {'fused' if big else 'pair'}, {'grid' if grid else 'continuous'}")
    a = agg.cpu().numpy()
    for k, name in enumerate(("sum", "mean", "min", "max", "std")):
        gates.check(name, a[:, k * H:(k + 1) * H], oagg[:, k * H:(k + 1) * H], FP32_FWD_TOL)
    f = fused.cpu().numpy()
    gates.check("dP", f[:, :H], odP, FP32_GRAD_TOL)
    gates.check("dQ", f[:, H:], odQ, FP32_GRAD_TOL)
    centre = int(b.node_off[len(STARS) - 1])                 # the first 254-leaf star's centre
    gates.check("dP centre", f[centre, :H], odP[centre], FP32_GRAD_TOL)
    gates.assert_all()


def _model_workload(big: bool, F: int, H: int, L: int, seed: int = 52):
    d = oracle.Dims(H=H, L=L, F=F)
    gs = _set(big, seed)
    gs.y = synth.uniform_targets(seed + 1, 0, gs.n_graphs, 1.0, 10.0)
    if F:
        gs.eattr = synth.bond_features(seed + 2, gs, F, -1.0, 1.0)
    return d, gs, synth.init_params(seed + 3, H, L, F=F)


@pytest.mark.parametrize("precision,F,big,recompute",
                         [(0, 0, False, False), (0, 4, False, False), (1, 0, False, False), (1, 4, False, False),
                          (0, 0, True, False), (1, 0, True, False), (0, 0, False, True), (1, 4, False, True),
                          (0, 0, True, True)],
                         ids=["fp32", "fp32-bonds", "bf16", "bf16-bonds", "fp32-fused", "bf16-fused",
                              "fp32-recompute", "bf16-bonds-recompute", "fp32-fused-recompute"])
def test_model_high_degree_vs_oracle(tmp_path, precision, F, big, recompute):
    """Per-layer recompute (the aggregates are dropped after the forward and
    recomputed in the backward) takes the stored-statistics branch of the
    FP32 backward and the shared-buffer path of the BF16 one."""
    H, L = (8, 2) if big else (32, 2)
    d, gs, p = _model_workload(big, F, H, L)
    path, ost = write_both(gs, str(tmp_path))
    import paper_2207_11333_gb300 as g
    st = g.Store(path)
    delta = st.delta()
    ctx = context(H, L, gs.n_graphs, gs.n_nodes, gs.n_edges, delta, precision=precision, F=F, recompute=recompute)
    ctx.set_params(p)
    ids = np.arange(gs.n_graphs)
    b = ctx.collate(st, ids)
    ob = oracle.collate(ost, ids, delta)
    assert ob.deg.max() == 254
    pred = torch.empty(b.n_graphs, device="cuda")
    ctx.forward(b, pred, train=True)
    acts = ctx.activations(b)
    ctx.backward(b)
    grads = ctx.get_grads()
    ctx.check()
    opred, oxs, _, _ = oracle.forward(d, p.astype(np.float64), ob, want_layers=True)
    _, ograd, _, _ = oracle.backward(d, p.astype(np.float64), ob)
    gv, ov = oracle.split_params(d, grads), oracle.split_params(d, ograd)
    gates = Gates(f"high-degree model, {'bf16' if precision else 'fp32'}, F = {F}, {'fused' if big else 'pair'}, "
                  f"recompute = {recompute}")
    if precision == 0:
        gates.check("pred", pred.cpu().numpy(), opred, FP32_FWD_TOL)
        for l in range(1, L + 1):
            gates.check(f"x{l}", acts[l], oxs[l], FP32_FWD_TOL)
        for k in ov:
            gates.check(k, gv[k], ov[k], FP32_GRAD_TOL)
    else:
        gates.check("pred", pred.cpu().numpy(), opred, BF16_FWD_TOL)
        for l in range(1, L + 1):
            gates.check(f"x{l}", acts[l], oxs[l], BF16_FWD_TOL)
        bound = bf16_grad_bound(L, residual_kappa(opred, ob.y))
        for k in ov:
            gates.check(k, gv[k], ov[k], bound, elementwise=False)
    gates.assert_all()
