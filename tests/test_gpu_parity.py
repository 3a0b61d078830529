"""The CUDA training step against the FP64 oracle on the 64-graph parity workload
(H = 32, L = 2) and ragged variants: forward within 1e-5, gradients within 1e-4
(FP32 path; both normwise and max elementwise relative, the elementwise error
floored at 1e-3 of the tensor's largest entry), Adam step, graph-captured step
== eager step."""
import numpy as np
import pytest
import torch

import oracle
import synth
import workloads
from gpu_common import context, oracle_step, write_both
from helpers import FP32_FWD_TOL as FWD_TOL, FP32_GRAD_TOL as GRAD_TOL, Gates, rel_norm

pytestmark = pytest.mark.gpu


def _setup(tmp_path, G=64, lo=5, hi=30, H=32, L=2, recompute=False):
    import paper_2207_11333_gb300 as g
    d, gs, delta, student = workloads.small_parity(G=G, lo=lo, hi=hi, H=H, L=L)
    path, ost = write_both(gs, str(tmp_path))
    st = g.Store(path)
    ctx = context(H, L, G, int(gs.n_nodes), int(gs.n_edges), delta, recompute=recompute)
    ctx.set_params(student)
    ids = np.arange(G)
    b = ctx.collate(st, ids)
    ob = oracle.collate(ost, ids, delta)
    return d, ctx, st, b, ob, student


@pytest.mark.parametrize("recompute", [False, True])
def test_forward_backward_step_parity(tmp_path, recompute):
    d, ctx, st, b, ob, student = _setup(tmp_path, recompute=recompute)
    pred = torch.empty(b.n_graphs, device="cuda")
    ctx.forward(b, pred, train=True)
    acts = ctx.activations(b)
    loss_acc = torch.zeros(3, dtype=torch.float64, device="cuda")
    ctx.backward(b, None, loss_acc)
    grads = ctx.get_grads()
    ctx.step(1e-3)
    new_params = ctx.get_params()
    ctx.check()

    opred, oxs, _, _ = oracle.forward(d, student.astype(np.float64), ob, want_layers=True)
    loss, ograd, _, oth = oracle_step(d, student, ob)
    gates = Gates(f"parity workload, recompute = {recompute}")
    gates.check("pred", pred.cpu().numpy(), opred, FWD_TOL)
    for l in range(d.L + 1):
        gates.check(f"x{l}", acts[l], oxs[l], FWD_TOL)
    la = loss_acc.cpu().numpy()
    assert abs(la[0] / la[2] - loss) < FWD_TOL * loss and la[2] == b.n_graphs
    assert abs(la[1] / la[2] - np.mean(np.abs(opred - ob.y))) < 1e-5 * la[1] / la[2]
    gv, ov = oracle.split_params(d, grads), oracle.split_params(d, ograd)
    for k in ov:
        gates.check(k, gv[k], ov[k], GRAD_TOL)
    gates.check("step", new_params - student, oth - student, 1e-3, elementwise=False)
    gates.check("params", new_params, oth, FWD_TOL)
    gates.assert_all()


# the last two batches have more than 2 x 152 x 128 edges, so the aggregation
# backward runs fused over chunks of whole graphs; in the last one most graphs
# have more edges than a chunk keeps in shared memory (the device-memory branch)
@pytest.mark.parametrize("G,lo,hi,H,L", [(1, 5, 5, 8, 1), (7, 3, 51, 16, 3), (33, 1, 80, 24, 2),
                                         (900, 3, 60, 16, 2), (400, 60, 120, 8, 1)])
def test_ragged_shapes(tmp_path, G, lo, hi, H, L):
    d, ctx, st, b, ob, student = _setup(tmp_path, G=G, lo=lo, hi=hi, H=H, L=L)
    pred = torch.empty(b.n_graphs, device="cuda")
    ctx.forward(b, pred, train=True)
    ctx.backward(b)
    grads = ctx.get_grads()
    ctx.check()
    loss, ograd, opred, _ = oracle_step(d, student, ob)
    gates = Gates(f"ragged G = {G}, atoms {lo}-{hi}, H = {H}, L = {L}")
    gates.check("pred", pred.cpu().numpy(), opred, FWD_TOL)
    gv, ov = oracle.split_params(d, grads), oracle.split_params(d, ograd)
    for k in ov:
        gates.check(k, gv[k], ov[k], GRAD_TOL)
    gates.assert_all()


def test_captured_train_step_matches_eager(tmp_path):
    d, ctx, st, b, ob, student = _setup(tmp_path)
    ctx.forward(b, train=True)
    ctx.backward(b)
    ctx.step(1e-3)
    eager = ctx.get_params()
    ctx.set_params(student)
    ctx.reset_optimizer()
    b = ctx.collate(st, np.arange(64))
    acc = torch.zeros(3, dtype=torch.float64, device="cuda")
    ctx.train_step(b, 1e-3, acc)
    captured = ctx.get_params()
    assert np.array_equal(eager, captured)
    # replay on another batch of the same bucket, then redo that step eagerly
    ckpt = str(tmp_path / "after1.bin")
    ctx.save(ckpt)
    ids = np.arange(64)[::-1].copy()
    ctx.train_step(ctx.collate(st, ids), 1e-3, acc)
    replay = ctx.get_params()
    ctx.load(ckpt)
    b = ctx.collate(st, ids)
    ctx.forward(b, train=True)
    ctx.backward(b)
    ctx.step(1e-3)
    assert np.array_equal(ctx.get_params(), replay)
    ctx.check()


def test_profiled_step_matches_and_times_phases(tmp_path):
    """With profiling on, train_step replays a graph with event-record nodes
    around every phase: same parameters bit for bit, every phase timed."""
    d, ctx, st, b, ob, student = _setup(tmp_path)
    acc = torch.zeros(3, dtype=torch.float64, device="cuda")
    ctx.train_step(b, 1e-3, acc)
    plain = ctx.get_params()
    ctx.set_params(student)
    ctx.reset_optimizer()
    ctx.profile(True)
    ctx.profile_read()
    b = ctx.collate(st, np.arange(64))
    ctx.train_step(b, 1e-3, acc)
    ph = ctx.profile_read()
    ctx.profile(False)
    assert np.array_equal(ctx.get_params(), plain)
    for k in ("collate", "embed", "gemm", "agg_fwd", "agg_bwd", "head", "embed_bwd", "adam"):
        assert ph[k][0] > 0 and ph[k][1] > 0, (k, ph[k])
    assert ph["gemm"][1] == 6 * d.L  # message, update and four backward GEMMs per layer
    ctx.check()


def test_kernel_timeline_of_a_train_step(tmp_path):
    """The kernel timeline records every launch of a collated train step in
    order (FP32 path here: collation, embedding, per-layer GEMMs and
    aggregations, head, backward, embedding gradient, optimiser, then the
    step-end marker), with non-decreasing device times, and nothing once
    disabled."""
    import paper_2207_11333_gb300 as g
    d, ctx, st, b, ob, student = _setup(tmp_path)
    acc = torch.zeros(3, dtype=torch.float64, device="cuda")
    ctx.timeline_enable(1024)
    try:
        ctx.timeline_read()
        b = ctx.collate(st, np.arange(64))
        ctx.train_step(b, 1e-3, acc)
        ids, t = ctx.timeline_read()
        names = [g.KERNELS[int(i)] for i in ids]
        assert names[:2] == ["collate", "embed"]    # 64 graphs: collated in one launch
        assert names[-3:] == ["embed_bwd", "adam", "step_end"]
        assert names.count("agg_fwd") == d.L and names.count("agg_bwd_edge") == d.L
        assert names.count("head_graph") == 1 and names.count("head_grad") == 1
        assert names.count("gemm_simt") == 6 * d.L
        assert np.all(np.diff(t) >= 0)
        ctx.timeline_read()
    finally:
        ctx.timeline_enable(0)
    ctx.train_step(ctx.collate(st, np.arange(64)), 1e-3, acc)
    with pytest.raises(g.GcnnError):
        ctx.timeline_read()
    ctx.check()


def test_checkpoint_resume_bitwise(tmp_path):
    d, ctx, st, b, ob, student = _setup(tmp_path)
    rng = np.random.default_rng(0)
    orders = [rng.permutation(64)[:48] for _ in range(4)]
    for o in orders[:2]:
        ctx.train_step(ctx.collate(st, o), 1e-3)
    ckpt = str(tmp_path / "c.bin")
    ctx.save(ckpt)
    for o in orders[2:]:
        ctx.train_step(ctx.collate(st, o), 1e-3)
    straight = ctx.get_params()
    ctx.set_params(student)
    ctx.reset_optimizer()
    ctx.load(ckpt)
    for o in orders[2:]:
        ctx.train_step(ctx.collate(st, o), 1e-3)
    assert np.array_equal(ctx.get_params(), straight)


def test_errors_are_reported(tmp_path):
    import paper_2207_11333_gb300 as g
    d, ctx, st, b, ob, student = _setup(tmp_path)
    b2 = ctx.collate(st, np.arange(10))
    with pytest.raises(g.GcnnError, match="ESTATE"):
        ctx.backward(b2)
    with pytest.raises(g.GcnnError, match="EINVAL"):
        g.Context(g.make_config(30, 2, 4, 100, 100, delta=1.0))       # hidden not a multiple of 8
    with pytest.raises(g.GcnnError, match="EINVAL"):
        ctx.set_params(np.zeros(5, np.float32))


def test_ffma_peak_is_plausible():
    """The FP32 FFMA probe (the roofline of the FP32 GEMM path) reports a rate
    between a quarter of and just above 152 SMs x 128 lanes x 2 FLOP x 2.07 GHz
    (80.5 TFLOP/s); iters < 1 is rejected."""
    import paper_2207_11333_gb300 as g
    t = g.ffma_peak(2048)
    assert 20.0 < t < 85.0, t
    with pytest.raises(g.GcnnError, match="EINVAL"):
        g.ffma_peak(0)
