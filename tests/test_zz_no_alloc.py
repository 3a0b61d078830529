"""gcnn_op_aggregate_bwd_noalloc: the aggregation backward for callers that cannot
allocate device memory (its scratch is a fixed array inside the library).

Called through the C ABI and compared with gcnn_op_aggregate_bwd, which takes a
caller-allocated scratch buffer, on two consecutive calls with different
graphs, so that contents left in the shared array by the first call cannot
leak into the second.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import oracle_batch, rel_norm

pytestmark = pytest.mark.gpu


def _case(seed, G, lo, hi, H):
    gs = synth.molecules_uniform(seed, G, lo, hi)
    _, b, _ = oracle_batch(gs)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    gen = torch.Generator(device="cuda").manual_seed(seed)
    PQ = torch.randn(b.N, 2 * H, device="cuda", generator=gen)
    dagg = torch.randn(b.N, 5 * H, device="cuda", generator=gen)
    return b, dev(b.row_ptr), dev(b.col), dev(b.rev), PQ, dagg


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_matches_caller_scratch_twice():
    import paper_2207_11333_gb300 as g
    lib = g.lib
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seed, G, lo, hi, H in [(31, 40, 5, 40, 64), (32, 25, 3, 20, 32)]:
        b, rp, col, rev, PQ, dagg = _case(seed, G, lo, hi, H)
        agg = torch.empty(b.N, 5 * H, device="cuda")
        assert lib.gcnn_op_aggregate_fwd(b.N, H, _p(rp), _p(col), _p(PQ), _p(agg), 1e-5, stream) == 0
        ref = torch.empty(b.N, 2 * H, device="cuda")
        scratch = torch.empty(b.E * H, device="cuda")
        assert lib.gcnn_op_aggregate_bwd(b.N, b.E, H, _p(rp), _p(col), _p(rev), _p(PQ), _p(agg), _p(dagg),
                                         _p(ref), _p(scratch), 1e-5, stream) == 0
        out = torch.full((b.N, 2 * H), float("nan"), device="cuda")
        rc = lib.gcnn_op_aggregate_bwd_noalloc(b.N, b.E, H, _p(rp), _p(col), _p(rev), _p(PQ), _p(agg),
                                               _p(dagg), _p(out), 1e-5, stream)
        assert rc == 0, lib.gcnn_last_error()
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert rel_norm(out.cpu().numpy(), ref.cpu().numpy()) < 1e-6


def test_noalloc_rejects_oversized_scratch():
    import paper_2207_11333_gb300 as g
    lib = g.lib
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    dummy = torch.zeros(16, device="cuda")
    rc = lib.gcnn_op_aggregate_bwd_noalloc(4, (1 << 22) // 64 + 1, 64, _p(dummy), _p(dummy), _p(dummy), _p(dummy),
                                           _p(dummy), _p(dummy), _p(dummy), 1e-5, stream)
    assert rc == -1
    assert b"exceeds the fixed scratch" in lib.gcnn_last_error()
