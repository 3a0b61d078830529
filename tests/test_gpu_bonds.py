"""Bond features in the message (m_ij = W_M [x_i ; x_j ; e_ij] + b_M; Sec. 3.1 bond
properties, Table 1 edge attributes): the CUDA path against the FP64 oracle on
molecules with F = 4 features per bond -- collation of the features bit-exact,
forward within 1e-5 and gradients (the bond rows included) within 1e-4 on the
FP32 path (normwise and elementwise), forward within 2e-2 and gradients within
the derived BF16 bound on the BF16 path; the host-staged collation
equals the device-resident one; mismatched feature counts are refused."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_common import context, oracle_step, write_both
from helpers import FP32_FWD_TOL, FP32_GRAD_TOL, Gates, bf16_grad_bound, rel_norm, residual_kappa

pytestmark = pytest.mark.gpu

F = 4


def _workload(G=64, lo=5, hi=30, H=32, L=2):
    d = oracle.Dims(H=H, L=L, F=F)
    gs = synth.molecules_uniform(41, G, lo, hi)
    gs.eattr = synth.bond_features(42, gs, F, -1.0, 1.0)
    st = oracle.store_from_arrays(gs.node_ptr, gs.edge_ptr, gs.types, gs.edges, gs.y, gs.eattr)
    delta = oracle.delta_of(st)
    b = oracle.collate(st, np.arange(G), delta)
    teacher = synth.init_params(43, H, L, F=F).astype(np.float64)
    gs.y = (oracle.forward(d, teacher, b) + synth.normal(44, 0, G, 0.05)).astype(np.float32)
    return d, gs, delta, synth.init_params(45, H, L, F=F)


def _setup(tmp_path, precision=0, recompute=False, resident=True, **kw):
    import paper_2207_11333_gb300 as g
    d, gs, delta, student = _workload(**kw)
    path, ost = write_both(gs, str(tmp_path))
    st = g.Store(path)
    assert st.edge_features == F
    if resident:
        st.to_device()
    ctx = context(d.H, d.L, gs.n_graphs, gs.n_nodes, gs.n_edges, delta, recompute=recompute,
                  precision=precision, F=F)
    ctx.set_params(student)
    ids = np.arange(gs.n_graphs)
    return d, g, ctx, st, ctx.collate(st, ids), oracle.collate(ost, ids, delta), student


@pytest.mark.parametrize("resident", [True, False], ids=["resident", "staged"])
def test_bond_features_collated_bit_exact(tmp_path, resident):
    d, g, ctx, st, b, ob, _ = _setup(tmp_path, resident=resident)
    ea = b.tensor("edge_attr").cpu().numpy()
    assert ea.shape == (ob.E, F)
    assert np.array_equal(ea, ob.eattr)
    ex = b.export()
    assert np.array_equal(ex["col"], ob.col) and np.array_equal(ex["rev"], ob.rev)


@pytest.mark.parametrize("recompute", [False, True])
def test_fp32_step_with_bond_features_matches_oracle(tmp_path, recompute):
    d, g, ctx, st, b, ob, student = _setup(tmp_path, recompute=recompute)
    pred = torch.empty(b.n_graphs, device="cuda")
    ctx.forward(b, pred, train=True)
    acts = ctx.activations(b)
    ctx.backward(b)
    grads = ctx.get_grads()
    ctx.check()
    opred, oxs, _, _ = oracle.forward(d, student.astype(np.float64), ob, want_layers=True)
    loss, ograd, _, oth = oracle_step(d, student, ob)
    gates = Gates(f"bond features F = {F}, recompute = {recompute}")
    gates.check("pred", pred.cpu().numpy(), opred, FP32_FWD_TOL)
    for l in range(d.L + 1):
        gates.check(f"x{l}", acts[l], oxs[l], FP32_FWD_TOL)
    gv, ov = oracle.split_params(d, grads), oracle.split_params(d, ograd)
    for k in ov:
        gates.check(k, gv[k], ov[k], FP32_GRAD_TOL)
    assert any(k.startswith("edge_w") for k in ov)
    gates.assert_all()


def test_captured_train_step_with_bond_features(tmp_path):
    """The captured step (forward, backward, AdamW) moves the parameters as the oracle's."""
    d, g, ctx, st, b, ob, student = _setup(tmp_path)
    acc = torch.zeros(3, dtype=torch.float64, device="cuda")
    ctx.train_step(b, 1e-3, acc)
    ctx.check()
    loss, _, _, oth = oracle_step(d, student, ob)
    la = acc.cpu().numpy()
    assert abs(la[0] / la[2] - loss) < 1e-5 * loss
    new = ctx.get_params()
    assert rel_norm(new - student, oth - student) < 1e-3
    assert rel_norm(new, oth) < 1e-5


def test_bf16_step_with_bond_features(tmp_path):
    d, g, ctx, st, b, ob, student = _setup(tmp_path, precision=1)
    pred = torch.empty(b.n_graphs, device="cuda")
    ctx.forward(b, pred, train=True)
    ctx.backward(b)
    grads = ctx.get_grads()
    ctx.check()
    opred = oracle.forward(d, student.astype(np.float64), ob)
    _, ograd, _, _ = oracle_step(d, student, ob)
    assert rel_norm(pred.cpu().numpy(), opred) < 2e-2
    gv, ov = oracle.split_params(d, grads), oracle.split_params(d, ograd)
    gates = Gates("bond features, bf16")
    bound = bf16_grad_bound(d.L, residual_kappa(opred, ob.y))
    for k in ov:
        gates.check(k, gv[k], ov[k], bound, elementwise=False)
    gates.assert_all()


def test_feature_count_mismatch_is_refused(tmp_path):
    import paper_2207_11333_gb300 as g
    d, gs, delta, student = _workload(G=8)
    path, _ = write_both(gs, str(tmp_path))
    st = g.Store(path)
    plain = context(d.H, d.L, gs.n_graphs, gs.n_nodes, gs.n_edges, delta)
    with pytest.raises(g.GcnnError, match="EINVAL"):
        plain.collate(st, np.arange(8))
    with_bonds = context(d.H, d.L, gs.n_graphs, gs.n_nodes, gs.n_edges, delta, F=F)
    with pytest.raises(g.GcnnError, match="EINVAL"):
        g.Server(with_bonds, n_slots=1, buckets=(1024,), max_graphs=64)
