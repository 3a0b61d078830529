"""Full model size (H = 200, L = 6, head 200-200-1) on a 256-graph slice of the
200k-graph training workload: per-layer forward and per-tensor gradient errors of
the FP32 and BF16 paths against the FP64 oracle.  FP32: forward <= 1e-5, gradients
<= 1e-4, normwise and elementwise; BF16: forward <= 2e-2, gradients within the
BF16 error bound derived in tests/helpers.py (bf16_grad_bound)."""
import json

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_common import context, write_both
from helpers import (BF16_FWD_TOL, FP32_FWD_TOL, FP32_GRAD_TOL, Gates, bf16_grad_bound, rel_norm,
                     residual_kappa)

pytestmark = pytest.mark.gpu

H, L, G = 200, 6, 256


@pytest.fixture(scope="module")
def reference(tmp_path_factory):
    gs = synth.molecules_lognormal(10, 200_000).subset(np.arange(G))
    gs.y = synth.uniform_targets(17, 0, G, 1.0, 10.0)
    path, ost = write_both(gs, str(tmp_path_factory.mktemp("full")))
    delta = oracle.delta_of(ost)
    ob = oracle.collate(ost, np.arange(G), delta)
    d = oracle.Dims(H=H, L=L)
    p = synth.init_params(3, H, L)
    opred, oxs, _, _ = oracle.forward(d, p.astype(np.float64), ob, want_layers=True)
    oloss, ograd, _, _ = oracle.backward(d, p.astype(np.float64), ob)
    return path, delta, ob, d, p, opred, oxs, oloss, ograd


@pytest.mark.parametrize("precision", [0, 1], ids=["fp32", "bf16"])
def test_full_size_layer_and_gradient_errors(reference, precision):
    import paper_2207_11333_gb300 as g
    path, delta, ob, d, p, opred, oxs, oloss, ograd = reference
    st = g.Store(path)
    ctx = context(H, L, G, ob.N, ob.E, delta, precision=precision)
    ctx.set_params(p)
    b = ctx.collate(st, np.arange(G))
    pred = torch.empty(G, device="cuda")
    ctx.forward(b, pred, train=True)
    acts = ctx.activations(b)
    ctx.backward(b)
    grads = ctx.get_grads()
    ctx.check()
    layer_err = [rel_norm(acts[l], oxs[l]) for l in range(1, L + 1)]
    pred_err = rel_norm(pred.cpu().numpy(), opred)
    gv, ov = oracle.split_params(d, grads), oracle.split_params(d, ograd)
    grad_err = {k: rel_norm(gv[k], ov[k]) for k in ov}
    print(json.dumps({"precision": "bf16" if precision else "fp32", "pred": pred_err, "layers": layer_err,
                      "grads": grad_err}))
    gates = Gates(f"full size H = {H}, L = {L}, {'bf16' if precision else 'fp32'}")
    if precision:
        gates.check("pred", pred.cpu().numpy(), opred, BF16_FWD_TOL)
        for l in range(1, L + 1):
            gates.check(f"x{l}", acts[l], oxs[l], BF16_FWD_TOL)
        bound = bf16_grad_bound(L, residual_kappa(opred, ob.y))
        for k in ov:
            gates.check(k, gv[k], ov[k], bound, elementwise=False)
    else:
        gates.check("pred", pred.cpu().numpy(), opred, FP32_FWD_TOL)
        for l in range(1, L + 1):
            gates.check(f"x{l}", acts[l], oxs[l], FP32_FWD_TOL)
        for k in ov:
            gates.check(k, gv[k], ov[k], FP32_GRAD_TOL)
    gates.assert_all()
