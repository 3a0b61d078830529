"""gcnn_op_aggregate_bwd_noalloc: the aggregation backward for callers that cannot
allocate device memory (its per-edge scratch is a fixed array inside the library).

Called through the C ABI on two consecutive calls with different graphs and
compared with gcnn_op_aggregate_bwd (the same backward with a caller-allocated
scratch buffer) and with the FP64 oracle's per-edge gradients summed per node
(oracle_aggregate_bwd_op), at the FP32 gradient gate of the other tests.  A
call whose scratch need is exactly the array's size (n_edges * hidden = 2^22)
is accepted and correct; one float more is refused.  A call that leaves NaN in
the shared array (its incoming gradient is NaN) is followed by a smaller call,
which must not see them: it reads only slots it has written itself (and the
entry point clears its part before it starts).  This file is collected last
on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import FP32_GRAD_TOL, Gates, custom_set, oracle_batch, rel_norm

pytestmark = pytest.mark.gpu

LIMIT = 1 << 22   # floats in the library's fixed scratch array


def _case(b, H, seed):
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    gen = torch.Generator(device="cuda").manual_seed(seed)
    PQ = torch.randn(b.N, 2 * H, device="cuda", generator=gen)
    dagg = torch.randn(b.N, 5 * H, device="cuda", generator=gen)
    return dev(b.row_ptr), dev(b.col), dev(b.rev), PQ, dagg


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _forward(lib, b, H, rp, col, PQ):
    agg = torch.empty(b.N, 5 * H, device="cuda")
    assert lib.gcnn_op_aggregate_fwd(b.N, H, _p(rp), _p(col), _p(PQ), _p(agg), 1e-5, _stream()) == 0
    return agg


def _noalloc(lib, b, H, rp, col, rev, PQ, agg, dagg):
    out = torch.full((b.N, 2 * H), float("nan"), device="cuda")
    rc = lib.gcnn_op_aggregate_bwd_noalloc(b.N, b.E, H, _p(rp), _p(col), _p(rev), _p(PQ), _p(agg), _p(dagg),
                                           _p(out), 1e-5, _stream())
    assert rc == 0, lib.gcnn_last_error()
    return out


def _oracle_dPQ(b, H, PQ, dagg):
    """dP_i = sum of dL/dm over node i's row, dQ_j = sum over the edges leaving j (FP64)."""
    pq = PQ.cpu().numpy().astype(np.float64)
    dst = np.repeat(np.arange(b.N), b.deg)
    m = pq[dst, :H] + pq[b.col, H:]
    agg = oracle.aggregate_op(b.row_ptr, m)
    dm = oracle.aggregate_bwd_op(b.row_ptr, m, agg, dagg.cpu().numpy().astype(np.float64))
    out = np.zeros((b.N, 2 * H))
    np.add.at(out[:, :H], dst, dm)
    np.add.at(out[:, H:], b.col, dm)
    return out


def test_noalloc_matches_caller_scratch_and_oracle_twice():
    import paper_2207_11333_gb300 as g
    lib = g.lib
    gates = Gates("no-allocation aggregation backward")
    for seed, G, lo, hi, H in [(31, 40, 5, 40, 64), (32, 25, 3, 20, 32)]:
        _, b, _ = oracle_batch(synth.molecules_uniform(seed, G, lo, hi))
        rp, col, rev, PQ, dagg = _case(b, H, seed)
        agg = _forward(lib, b, H, rp, col, PQ)
        ref = torch.empty(b.N, 2 * H, device="cuda")
        scratch = torch.empty(b.E * H, device="cuda")
        assert lib.gcnn_op_aggregate_bwd(b.N, b.E, H, _p(rp), _p(col), _p(rev), _p(PQ), _p(agg), _p(dagg),
                                         _p(ref), _p(scratch), 1e-5, _stream()) == 0
        out = _noalloc(lib, b, H, rp, col, rev, PQ, agg, dagg)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        gates.check(f"vs op, seed {seed}", out.cpu().numpy(), ref.cpu().numpy(), 1e-6)
        gates.check(f"vs oracle, seed {seed}", out.cpu().numpy(), _oracle_dPQ(b, H, PQ, dagg), FP32_GRAD_TOL)
    gates.assert_all()


def test_noalloc_at_the_size_limit_and_after_stale_contents():
    """64 cycles of 128 atoms: 16,384 directed edges, hidden 256, so the call
    needs exactly the 2^22 floats of the array.  It runs with a NaN incoming
    gradient first (every slot of the array then holds NaN), then with a finite
    one on the same graphs, then on a smaller batch: both later results are
    finite and match the allocating entry point and the oracle."""
    import paper_2207_11333_gb300 as g
    lib = g.lib
    H = 256
    ring = [(k, (k + 1) % 128) for k in range(128)]
    _, b, _ = oracle_batch(custom_set([([k % 7 for k in range(128)], ring)] * 64))
    assert b.E * H == LIMIT
    rp, col, rev, PQ, dagg = _case(b, H, 41)
    agg = _forward(lib, b, H, rp, col, PQ)
    poisoned = _noalloc(lib, b, H, rp, col, rev, PQ, agg, torch.full_like(dagg, float("nan")))
    torch.cuda.synchronize()
    assert torch.isnan(poisoned).all()
    gates = Gates("no-allocation backward at 2^22 floats")
    out = _noalloc(lib, b, H, rp, col, rev, PQ, agg, dagg)
    ref = g.aggregate_bwd(PQ, agg, dagg, rp, col, rev)
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()
    gates.check("limit vs op", out.cpu().numpy(), ref.cpu().numpy(), 1e-6)
    gates.check("limit vs oracle", out.cpu().numpy(), _oracle_dPQ(b, H, PQ, dagg), FP32_GRAD_TOL)
    _noalloc(lib, b, H, rp, col, rev, PQ, agg, torch.full_like(dagg, float("nan")))
    _, b2, _ = oracle_batch(synth.molecules_uniform(33, 30, 5, 30))
    rp2, col2, rev2, PQ2, dagg2 = _case(b2, 64, 42)
    agg2 = _forward(lib, b2, 64, rp2, col2, PQ2)
    out2 = _noalloc(lib, b2, 64, rp2, col2, rev2, PQ2, agg2, dagg2)
    ref2 = g.aggregate_bwd(PQ2, agg2, dagg2, rp2, col2, rev2)
    torch.cuda.synchronize()
    assert torch.isfinite(out2).all()
    gates.check("after NaN vs op", out2.cpu().numpy(), ref2.cpu().numpy(), 1e-6)
    gates.check("after NaN vs oracle", out2.cpu().numpy(), _oracle_dPQ(b2, 64, PQ2, dagg2), FP32_GRAD_TOL)
    gates.assert_all()


def test_noalloc_rejects_oversized_scratch():
    import paper_2207_11333_gb300 as g
    lib = g.lib
    dummy = torch.zeros(16, device="cuda")
    rc = lib.gcnn_op_aggregate_bwd_noalloc(4, LIMIT // 64 + 1, 64, _p(dummy), _p(dummy), _p(dummy), _p(dummy),
                                           _p(dummy), _p(dummy), _p(dummy), 1e-5, _stream())
    assert rc == -1
    assert b"exceeds the fixed scratch" in lib.gcnn_last_error()
    assert rel_norm(dummy.cpu().numpy(), np.zeros(16)) == 0.0      # nothing was written
