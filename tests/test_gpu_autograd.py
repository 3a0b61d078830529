"""torch.autograd.Function wrappers of the aggregation and pooling kernels: forward
and backward against a plain PyTorch FP64 statement of the same ops (autograd of
scatter_reduce), directional finite differences, and the composed PNA layer against
the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import oracle_batch, rel_norm

pytestmark = pytest.mark.gpu


def _graph(seed=11, G=20, lo=3, hi=40):
    gs = synth.molecules_uniform(seed, G, lo, hi)
    _, b, delta = oracle_batch(gs)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return b, delta, dev(b.row_ptr), dev(b.col), dev(b.rev), dev(b.node_off.astype(np.int32)), dev(b.graph_id)


def _torch_aggregate(PQ, b, H, eps=1e-5):
    """The five aggregators by torch.scatter_reduce (FP64 reference)."""
    dst = torch.from_numpy(np.repeat(np.arange(b.N), np.diff(b.row_ptr))).long().to(PQ.device)
    src = torch.from_numpy(b.col.astype(np.int64)).to(PQ.device)
    m = PQ[dst, :H] + PQ[src, H:]
    idx = dst.unsqueeze(1).expand(-1, H)
    z = torch.zeros(b.N, H, dtype=PQ.dtype, device=PQ.device)
    s = z.scatter_reduce(0, idx, m, "sum", include_self=False)
    mean = z.scatter_reduce(0, idx, m, "mean", include_self=False)
    mn = z.scatter_reduce(0, idx, m, "amin", include_self=False)
    mx = z.scatter_reduce(0, idx, m, "amax", include_self=False)
    dev = m - mean[dst]
    var = z.index_add(0, dst, dev * dev) / torch.from_numpy(np.maximum(b.deg, 1)).to(PQ).unsqueeze(1)
    sd = torch.sqrt(torch.relu(var) + eps)
    has = torch.from_numpy((b.deg > 0).astype(np.float64)).to(PQ).unsqueeze(1)
    return torch.cat([s, mean, mn, mx, sd], 1) * has


def test_aggregate_function_matches_torch_fp64():
    from paper_2207_11333_gb300.autograd import aggregate
    b, delta, rp, col, rev, _, _ = _graph()
    H = 24
    gen = torch.Generator(device="cuda").manual_seed(0)
    PQ = torch.randn(b.N, 2 * H, device="cuda", generator=gen)
    W = torch.randn(b.N, 5 * H, device="cuda", generator=gen)
    x = PQ.clone().requires_grad_(True)
    (aggregate(x, rp, col, rev) * W).sum().backward()
    ref_x = PQ.double().clone().requires_grad_(True)
    ref = _torch_aggregate(ref_x, b, H)
    (ref * W.double()).sum().backward()
    assert rel_norm(aggregate(PQ, rp, col, rev).cpu().numpy(), ref.detach().cpu().numpy()) < 1e-6
    assert rel_norm(x.grad.cpu().numpy(), ref_x.grad.cpu().numpy()) < 1e-5


@pytest.mark.parametrize("G,lo,hi,H", [(20, 3, 40, 12), (900, 3, 60, 8), (400, 60, 120, 4)])
def test_aggregate_bwd_over_graphs_matches_pair(G, lo, hi, H):
    """gcnn_op_aggregate_bwd_graphs (fused over chunks of whole graphs once the
    batch has more than 2 x SMs x 128 edges; graphs above a chunk's shared-memory
    slots go through device memory) equals the edge + gather pair bitwise and
    the FP64 torch gradient, with a trailing graph of isolated atoms.  P holds odd
    and Q even multiples of 1/16, so every message P_i + Q_j is exact in FP32 and
    FP64 (both sides take the same min/max decisions, exact ties included, on a
    batch of tens of thousands of atoms) and never 0, the value torch's amax/amin
    reference starts from and would count as a tie."""
    import paper_2207_11333_gb300 as g
    gs = synth.molecules_uniform(17, G, lo, hi)
    _, b, delta = oracle_batch(gs)
    extra = 3                                              # one more graph: 3 atoms, no edges
    N = b.N + extra
    row_ptr = np.concatenate([b.row_ptr, np.full(extra, b.row_ptr[-1], np.int32)]).astype(np.int32)
    node_off = np.concatenate([b.node_off, [N]]).astype(np.int32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rp, col, rev, no = dev(row_ptr), dev(b.col), dev(b.rev), dev(node_off)
    gen = torch.Generator(device="cuda").manual_seed(4)
    k = torch.randint(-64, 64, (N, 2 * H), device="cuda", generator=gen).float()
    PQ = torch.cat([2 * k[:, :H] + 1, 2 * k[:, H:]], 1) / 16
    dagg = torch.randn(N, 5 * H, device="cuda", generator=gen)
    agg = g.aggregate_fwd(PQ, rp, col)
    pair = g.aggregate_bwd(PQ, agg, dagg, rp, col, rev)
    fused = g.aggregate_bwd(PQ, agg, dagg, rp, col, rev, node_off=no)
    torch.cuda.synchronize()
    assert torch.equal(pair, fused)
    bb = type("B", (), {})()
    bb.N, bb.row_ptr, bb.col = N, row_ptr, b.col
    bb.deg = np.diff(row_ptr)
    ref_x = PQ.double().clone().requires_grad_(True)
    (_torch_aggregate(ref_x, bb, H) * dagg.double()).sum().backward()
    assert rel_norm(fused.cpu().numpy(), ref_x.grad.cpu().numpy()) < 1e-5
    assert torch.count_nonzero(fused[b.N:]) == 0


def test_aggregate_function_ties_match_torch():
    """Identical sources (as from equal atom types) tie in min/max; the split matches torch."""
    from paper_2207_11333_gb300.autograd import aggregate
    b, delta, rp, col, rev, _, _ = _graph(seed=12)
    H = 8
    gen = torch.Generator(device="cuda").manual_seed(1)
    base = torch.randn(3, 2 * H, device="cuda", generator=gen)
    PQ = base[torch.from_numpy(np.arange(b.N) % 3).cuda()].contiguous()
    W = torch.randn(b.N, 5 * H, device="cuda", generator=gen)
    x = PQ.clone().requires_grad_(True)
    (aggregate(x, rp, col, rev) * W).sum().backward()
    ref_x = PQ.double().clone().requires_grad_(True)
    (_torch_aggregate(ref_x, b, H) * W.double()).sum().backward()
    assert rel_norm(x.grad.cpu().numpy(), ref_x.grad.cpu().numpy()) < 1e-5


def test_aggregate_directional_finite_differences():
    """Central differences along random directions, on the smooth aggregators (sum,
    mean, std with a large epsilon so sqrt(var + eps) has little curvature at step h);
    min/max are piecewise linear and pinned by the torch comparisons."""
    from paper_2207_11333_gb300.autograd import aggregate
    b, delta, rp, col, rev, _, _ = _graph(seed=13)
    H = 16
    gen = torch.Generator(device="cuda").manual_seed(2)
    PQ = torch.randn(b.N, 2 * H, device="cuda", generator=gen)
    W = torch.randn(b.N, 5 * H, device="cuda", generator=gen)
    W[:, 2 * H:4 * H] = 0.0
    x = PQ.clone().requires_grad_(True)
    eps = 1.0
    (aggregate(x, rp, col, rev, eps) * W).sum().backward()
    for k in range(5):
        V = torch.randn(b.N, 2 * H, device="cuda", generator=gen)
        h = 1e-3
        f = lambda t: (aggregate(t, rp, col, rev, eps).double() * W.double()).sum().item()
        fd = (f(PQ + h * V) - f(PQ - h * V)) / (2 * h)
        an = float((x.grad.double() * V.double()).sum())
        assert abs(fd - an) <= 2e-3 * abs(an) + 1e-2, (k, fd, an)


def test_mean_pool_function():
    from paper_2207_11333_gb300.autograd import mean_pool
    b, delta, rp, col, rev, node_off, gid = _graph(seed=14)
    H = 12
    gen = torch.Generator(device="cuda").manual_seed(3)
    X = torch.randn(b.N, H, device="cuda", generator=gen)
    W = torch.randn(b.G, H, device="cuda", generator=gen)
    x = X.clone().requires_grad_(True)
    (mean_pool(x, node_off, gid) * W).sum().backward()
    counts = torch.from_numpy(np.diff(b.node_off)).double().cuda()
    ref_x = X.double().clone().requires_grad_(True)
    ref = torch.zeros(b.G, H, dtype=torch.float64, device="cuda").index_add(0, gid.long(), ref_x) / counts[:, None]
    (ref * W.double()).sum().backward()
    assert rel_norm(mean_pool(X, node_off, gid).cpu().numpy(), ref.detach().cpu().numpy()) < 1e-6
    assert rel_norm(x.grad.cpu().numpy(), ref_x.grad.cpu().numpy()) < 1e-6


def test_composed_layer_against_oracle():
    """One PNA layer composed from torch matmuls and the Functions: the pooled-MSE
    gradients w.r.t. the layer's weights match the FP64 oracle."""
    from paper_2207_11333_gb300.autograd import aggregate, mean_pool
    H, L = 16, 1
    d = oracle.Dims(H=H, L=L)
    gs = synth.molecules_uniform(15, 12, 5, 25)
    gs.y = synth.uniform_targets(16, 0, 12, 1, 10)
    _, b, delta = oracle_batch(gs)
    p = synth.init_params(3, H, L)
    W = oracle.split_params(d, p.astype(np.float64))
    cu = lambda a, rg=False: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda", requires_grad=rg)
    ci = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    emb, msg_w, msg_b = cu(W["emb"]), cu(W["msg_w0"], True), cu(W["msg_b0"], True)
    upd_w, upd_b = cu(W["upd_w0"], True), cu(W["upd_b0"], True)
    w1, b1, w2, b2 = cu(W["w1"]), cu(W["b1"]), cu(W["w2"]), cu(W["b2"])
    x = emb[ci(b.types.astype(np.int64))]
    PQ = x @ msg_w + torch.cat([msg_b, torch.zeros_like(msg_b)])
    agg = aggregate(PQ, ci(b.row_ptr), ci(b.col), ci(b.rev))
    amp, att = ci(b.amp)[:, None], ci(b.att)[:, None]
    h = torch.relu(torch.cat([x, agg, agg * amp, agg * att], 1) @ upd_w + upd_b)
    g = mean_pool(h, ci(b.node_off.astype(np.int32)), ci(b.graph_id))
    pred = torch.relu(g @ w1 + b1) @ w2 + b2
    loss = torch.mean((pred - ci(b.y)) ** 2)
    loss.backward()
    oloss, ograd, _, _ = oracle.backward(d, p.astype(np.float64), b)
    og = oracle.split_params(d, ograd)
    assert abs(loss.item() - oloss) < 1e-5 * oloss
    for name, t in (("msg_w0", msg_w), ("msg_b0", msg_b), ("upd_w0", upd_w), ("upd_b0", upd_b)):
        assert rel_norm(t.grad.cpu().numpy(), og[name]) < 1e-4, name


def test_aggregate_function_with_graph_offsets():
    """The Function's backward over whole graphs (fused on a batch of 900 molecules)
    equals the pair's."""
    from paper_2207_11333_gb300.autograd import aggregate
    b, delta, rp, col, rev, node_off, _ = _graph(seed=18, G=900, lo=3, hi=60)
    H = 8
    gen = torch.Generator(device="cuda").manual_seed(6)
    PQ = torch.randn(b.N, 2 * H, device="cuda", generator=gen)
    W = torch.randn(b.N, 5 * H, device="cuda", generator=gen)
    x1 = PQ.clone().requires_grad_(True)
    x2 = PQ.clone().requires_grad_(True)
    (aggregate(x1, rp, col, rev) * W).sum().backward()
    (aggregate(x2, rp, col, rev, 1e-5, node_off) * W).sum().backward()
    assert torch.equal(x1.grad, x2.grad)
