"""gcnn_train_step_range: the collation of a range of the device-resident order
captured in the same CUDA graph as the training step.  Consecutive ranges
(the graph's collation nodes updated between launches, a smaller last batch
with a graph of its own, a return to the first range, and a new order
uploaded between two launches) give the parameters, loss sums and batches of
gcnn_collate_range + gcnn_train_step bit for bit."""
import numpy as np
import pytest
import torch

import workloads
from gpu_common import write_both

pytestmark = pytest.mark.gpu

RANGES = [(0, 64), (64, 64), (128, 64), (192, 64), (256, 44), (0, 64), (128, 64)]


def _trained(g, st, gs, delta, student, precision, ranged):
    G, H, L = 64, 32, 2
    ctx = g.Context(g.make_config(H, L, G, int(gs.n_nodes), int(gs.n_edges), delta=delta, precision=precision,
                                  head_hidden=H))
    ctx.set_params(student)
    ctx.set_order(st, np.random.default_rng(5).permutation(300))
    acc = torch.zeros(3, dtype=torch.float64, device="cuda")
    batches = []
    for k, (first, count) in enumerate(RANGES):
        if k == len(RANGES) - 2:   # a new order: the cached graph must read the new id list
            ctx.set_order(st, np.random.default_rng(6).permutation(300))
        if ranged:
            b = ctx.train_step_range(st, first, count, 1e-3, acc)
        else:
            b = ctx.collate_range(st, first, count)
            ctx.train_step(b, 1e-3, acc)
        batches.append(b.export())
    out = (ctx.get_params(), acc.cpu().numpy(), batches)
    ctx.check()
    ctx.close()
    return out


@pytest.mark.parametrize("precision", ["bf16", "fp32"])
def test_train_step_range_equals_collate_then_train_step(tmp_path, precision):
    import paper_2207_11333_gb300 as g
    _, gs, delta, student = workloads.small_parity(G=300, lo=5, hi=30, H=32, L=2)
    path, _ = write_both(gs, str(tmp_path))
    st = g.Store(path)
    st.to_device()
    prec = g.PREC_BF16 if precision == "bf16" else g.PREC_FP32
    p_ref, acc_ref, b_ref = _trained(g, st, gs, delta, student, prec, ranged=False)
    p_new, acc_new, b_new = _trained(g, st, gs, delta, student, prec, ranged=True)
    assert np.array_equal(p_ref, p_new)
    assert np.array_equal(acc_ref, acc_new)
    assert acc_new[2] == sum(c for _, c in RANGES)
    for x, y in zip(b_ref, b_new):
        assert x.keys() == y.keys()
        for k in x:
            assert np.array_equal(x[k], y[k]), k


def test_train_step_range_rejects_bad_ranges(tmp_path):
    import paper_2207_11333_gb300 as g
    _, gs, delta, student = workloads.small_parity(G=80, lo=5, hi=30, H=32, L=2)
    path, _ = write_both(gs, str(tmp_path))
    st = g.Store(path)
    st.to_device()
    ctx = g.Context(g.make_config(32, 2, 64, int(gs.n_nodes), int(gs.n_edges), delta=delta, head_hidden=32))
    ctx.set_params(student)
    with pytest.raises(g.GcnnError, match="ESTATE"):
        ctx.train_step_range(st, 0, 64, 1e-3)
    ctx.set_order(st, np.arange(80))
    with pytest.raises(g.GcnnError, match="EINVAL"):
        ctx.train_step_range(st, 40, 64, 1e-3)     # past the end of the order
    with pytest.raises(g.GcnnError, match="EINVAL"):
        ctx.train_step_range(st, 0, 80, 1e-3)      # more graphs than the context holds
    ctx.train_step_range(st, 16, 64, 1e-3)
    ctx.check()
    ctx.close()


def test_train_step_range_beyond_the_single_launch_collation(tmp_path):
    """Batches of more than 1024 graphs are collated by two launches: both of
    the graph's collation nodes move to the next range."""
    import paper_2207_11333_gb300 as g
    import synth
    n_total, G, H, L = 2400, 1100, 32, 1
    gs = synth.molecules_uniform(31, n_total, 2, 12)
    gs.y = synth.uniform_targets(32, 0, n_total, 1.0, 10.0)
    path, _ = write_both(gs, str(tmp_path))
    st = g.Store(path)
    st.to_device()
    delta = st.delta()
    student = synth.init_params(3, H, L)
    order = np.random.default_rng(33).permutation(n_total)
    res = []
    for ranged in (False, True):
        ctx = g.Context(g.make_config(H, L, G, int(gs.n_nodes), int(gs.n_edges), delta=delta, head_hidden=H))
        ctx.set_params(student)
        ctx.set_order(st, order)
        acc = torch.zeros(3, dtype=torch.float64, device="cuda")
        exports = []
        for first in (0, 1100, 0):
            if ranged:
                b = ctx.train_step_range(st, first, G, 1e-3, acc)
            else:
                b = ctx.collate_range(st, first, G)
                ctx.train_step(b, 1e-3, acc)
            exports.append(b.export())
        res.append((ctx.get_params(), acc.cpu().numpy(), exports))
        ctx.check()
        ctx.close()
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1], res[1][1])
    for x, y in zip(res[0][2], res[1][2]):
        for k in x:
            assert np.array_equal(x[k], y[k]), k
