"""BF16 tensor-core GEMM path (tcgen05) against the FP64 oracle: forward within
2e-2 relative (normwise) per output and per layer, predictions also
elementwise; gradients within the BF16 error bound derived in tests/helpers.py
(bf16_grad_bound: operand rounding along the GEMM chain plus ReLU / min-max
decision flips); the BF16 and FP32 paths agree to BF16 accuracy."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from gpu_common import oracle_step, write_both
from helpers import BF16_FWD_TOL, Gates, bf16_grad_bound, rel_norm, residual_kappa

pytestmark = pytest.mark.gpu


def _run(tmp_path, precision, G=64, lo=5, hi=30, H=32, L=2, recompute=False, serial=False):
    import paper_2207_11333_gb300 as g
    d, gs, delta, student = workloads.small_parity(G=G, lo=lo, hi=hi, H=H, L=L)
    path, ost = write_both(gs, str(tmp_path))
    st = g.Store(path)
    ctx = g.Context(g.make_config(H, L, G, int(gs.n_nodes), int(gs.n_edges), delta=delta, precision=precision,
                                  recompute=int(recompute), head_hidden=H, flags=g.FLAG_SERIAL if serial else 0))
    ctx.set_params(student)
    b = ctx.collate(st, np.arange(G))
    pred = torch.empty(G, device="cuda")
    ctx.forward(b, pred, train=True)
    acts = ctx.activations(b)
    ctx.backward(b)
    grads = ctx.get_grads()
    ctx.check()
    ob = oracle.collate(ost, np.arange(G), delta)
    return d, student, ob, pred.cpu().numpy(), acts, grads


# the case of 900 graphs has more than 2 x 152 x 128 edges: its aggregation
# backward runs fused over chunks of whole graphs and writes the BF16 [dP | dQ]
# operand there; at H = 256 the bias sums cover 2H = 512 columns, 16 groups of 32
# (13 at H = 200, the last one partly filled)
@pytest.mark.parametrize("G,lo,hi,H,L", [(64, 5, 30, 32, 2), (13, 3, 51, 200, 2), (150, 3, 51, 64, 3),
                                         (900, 3, 60, 32, 2), (40, 3, 30, 256, 1)])
def test_bf16_forward_and_gradients(tmp_path, G, lo, hi, H, L):
    import paper_2207_11333_gb300 as g
    d, student, ob, pred, acts, grads = _run(tmp_path, g.PREC_BF16, G, lo, hi, H, L)
    opred, oxs, _, _ = oracle.forward(d, student.astype(np.float64), ob, want_layers=True)
    _, ograd, _, _ = oracle_step(d, student, ob)
    gates = Gates(f"bf16 G = {G}, H = {H}, L = {L}")
    gates.check("pred", pred, opred, BF16_FWD_TOL)
    for l in range(1, d.L + 1):
        gates.check(f"x{l}", acts[l], oxs[l], BF16_FWD_TOL)
    gv, ov = oracle.split_params(d, grads), oracle.split_params(d, ograd)
    bound = bf16_grad_bound(d.L, residual_kappa(opred, ob.y))
    for k in ov:
        gates.check(k, gv[k], ov[k], bound, elementwise=False)
    gates.assert_all()


def test_bf16_matches_fp32_path(tmp_path):
    import paper_2207_11333_gb300 as g
    _, _, _, p16, a16, g16 = _run(tmp_path, g.PREC_BF16)
    _, _, _, p32, a32, g32 = _run(tmp_path, g.PREC_FP32)
    assert rel_norm(p16, p32) < BF16_FWD_TOL
    assert rel_norm(g16, g32) < bf16_grad_bound(2)


@pytest.mark.parametrize("G,hi", [(64, 30), (900, 60)])
def test_bf16_recompute_identical(tmp_path, G, hi):
    """Recompute (a one-stream backward) against the stored path, both with its
    default overlapped backward and on one stream: identical bit for bit."""
    import paper_2207_11333_gb300 as g
    _, _, _, p1, _, g1 = _run(tmp_path, g.PREC_BF16, G=G, lo=3, hi=hi, recompute=False)
    _, _, _, p2, _, g2 = _run(tmp_path, g.PREC_BF16, G=G, lo=3, hi=hi, recompute=True)
    _, _, _, p3, _, g3 = _run(tmp_path, g.PREC_BF16, G=G, lo=3, hi=hi, recompute=False, serial=True)
    assert np.array_equal(p1, p2) and np.array_equal(g1, g2)
    assert np.array_equal(p1, p3) and np.array_equal(g1, g3)


def test_overlapped_backward_matches_serial(tmp_path):
    """The BF16 backward's weight-gradient work on a second stream (default)
    gives the same gradients and parameters, bit for bit, as the serial step
    (GCNN_FLAG_SERIAL), over captured train steps and an eager backward: the
    weight-gradient GEMMs plan with the same CTA limit in both modes.  In the
    overlapped train steps the AdamW updates of layers L-1 .. 1 run on the
    second stream during the backward, the serial ones update everything at the
    end: the step counter and the parameters still agree."""
    import paper_2207_11333_gb300 as g
    G, H, L = 96, 64, 3
    d, gs, delta, student = workloads.small_parity(G=G, lo=3, hi=51, H=H, L=L)
    path, _ = write_both(gs, str(tmp_path))
    st = g.Store(path)
    res = []
    for flags in (0, g.FLAG_SERIAL):
        cfg = g.make_config(H, L, G, int(gs.n_nodes), int(gs.n_edges), delta=delta, precision=g.PREC_BF16,
                            flags=flags, head_hidden=H)
        ctx = g.Context(cfg)
        ctx.set_params(student)
        acc = torch.zeros(3, dtype=torch.float64, device="cuda")
        for k in range(3):
            ids = np.random.default_rng(k).permutation(G)
            ctx.train_step(ctx.collate(st, ids), 1e-3, acc)
        b = ctx.collate(st, np.arange(G))
        ctx.forward(b, train=True)
        ctx.backward(b)
        res.append((ctx.get_params(), ctx.get_grads(), acc.cpu().numpy()))
        ctx.check()
        ctx.close()
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1], res[1][1])
    assert np.array_equal(res[0][2], res[1][2])


def test_gemm_study_times_every_shape():
    """gcnn_gemm_study (measurement support) times the six GEMM shapes of a step
    under the planner's plan and under its search space, and the update shape
    against K; a bad size is refused."""
    import paper_2207_11333_gb300 as g
    rows = g.gemm_study(512, 32, 0)
    for name in g.GEMM_SHAPES:
        mine = [r for r in rows if r["shape"] == name]
        assert sum(r["planner"] for r in mine) == 1 and len(mine) > 1, name
        assert all(0.0 < r["us"] < 1e4 for r in mine)
    sweep = g.gemm_study(512, 32, 1)
    assert {r["BN"] for r in sweep} == {32, 64, 112, 128}
    assert all(r["shape"] == "update" and r["splits"] == 1 for r in sweep)
    with pytest.raises(g.GcnnError, match="EINVAL"):
        g.gemm_study(512, 30, 0)
