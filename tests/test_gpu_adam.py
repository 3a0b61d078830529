"""AdamW (Sec. 3.2, Fig. 3: the optimizer step; Sec. 5.1: AdamW) over several
steps against the FP64 oracle, with and without decoupled weight decay.

Each step t = 1..5 uses another batch and another learning rate.  Before the
step the test reads the context's parameters, Adam moments and step counter
(a checkpoint) and its gradients; after the step it reads them again and
compares them with oracle_adam applied to the same FP64-promoted state, step
number t, rate and decay.  So the moment updates, the bias corrections
1/(1 - beta^t) for t >= 2 and the decay are all compared, element by element,
for the eager step, the captured FP32 step and the captured BF16 step (whose
layers are updated on a third stream during the backward).  A second test runs
the whole trajectory on the oracle (its own gradients) and compares the
parameters after every step.

Gates, from the FP32 arithmetic of the same operations (unit roundoff
u = 2^-24), entry by entry: m within 4u and v within 6u of the magnitudes of
their two terms (b1 |m| + (1 - b1) |g|, and b2 v + (1 - b2) g^2: two products,
a square and a sum); the parameters within 4u |theta| (decay and update
subtracted) plus 16u of the update (the bias corrections, a square root, a
division and the rate) plus m's own error carried into the update by
lr c1 / (sqrt(v c2) + eps), which dominates where successive gradients change
sign and m nearly cancels; normwise, the parameters within 1e-6.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads
from gpu_common import write_both
from helpers import Gates

pytestmark = pytest.mark.gpu

STEPS = 5
RATES = (1e-3, 5e-4, 2e-3, 1e-3, 3e-4)
U32 = 2.0 ** -24


def _read_state(ctx, path):
    ctx.save(path)
    raw = np.fromfile(path, np.uint8)
    assert raw[:8].tobytes() == b"GCNNCKP1"
    P = int(raw[8:16].view("<i8")[0])
    t = int(raw[16:20].view("<i4")[0])
    body = raw[20:20 + 12 * P].view("<f4")
    return t, body[:P].copy(), body[P:2 * P].copy(), body[2 * P:].copy()


def _setup(tmp_path, wd, precision, H=32, L=2, G=64):
    import paper_2207_11333_gb300 as g
    d, gs, delta, student = workloads.small_parity(G=G, H=H, L=L)
    path, ost = write_both(gs, str(tmp_path))
    st = g.Store(path)
    ctx = g.Context(g.make_config(H, L, G, int(gs.n_nodes), int(gs.n_edges), delta=delta, precision=precision,
                                  head_hidden=H, weight_decay=wd))
    ctx.set_params(student)
    return d, g, ctx, st, ost, delta, student


@pytest.mark.parametrize("mode", ["eager", "captured-fp32", "captured-bf16"])
@pytest.mark.parametrize("wd", [0.0, 0.01])
def test_adamw_steps_match_oracle(tmp_path, wd, mode):
    d, g, ctx, st, ost, delta, student = _setup(tmp_path, wd, 1 if mode == "captured-bf16" else 0)
    ck = str(tmp_path / "state.bin")
    rng = np.random.default_rng(5)
    gates = Gates(f"AdamW, wd = {wd}, {mode}")
    for t in range(1, STEPS + 1):
        ids = rng.permutation(64)[:40 + 4 * t]
        lr = RATES[t - 1]
        t0, p0, m0, v0 = _read_state(ctx, ck)
        assert t0 == t - 1
        b = ctx.collate(st, ids)
        if mode == "eager":
            ctx.forward(b, train=True)
            ctx.backward(b)
            grads = ctx.get_grads()
            ctx.step(lr)
        else:
            ctx.train_step(b, lr)
            grads = ctx.get_grads()          # the backward overwrites them; AdamW leaves them
        ctx.check()
        t1, p1, m1, v1 = _read_state(ctx, ck)
        assert t1 == t
        th, m, v = p0.astype(np.float64), m0.astype(np.float64), v0.astype(np.float64)
        g64 = grads.astype(np.float64)
        oracle.adam(th, g64, m, v, t, lr=lr, wd=wd)
        upd = np.abs(th - p0.astype(np.float64) * (1.0 - lr * wd))
        s_m = 0.9 * np.abs(m0) + 0.1 * np.abs(g64)          # magnitudes of m's two terms
        gates.check_abs(f"m t={t}", m1 - m, s_m, 4 * U32)
        gates.check_abs(f"v t={t}", v1 - v, 0.999 * v0 + 0.001 * g64 * g64, 6 * U32)
        # theta: its own rounding, a dozen roundings of the update, and m's error
        # (4u of its terms, large against m where g changed sign) carried by
        # lr c1 / (sqrt(v c2) + eps) into the update
        c1, c2 = 1.0 / (1.0 - 0.9 ** t), 1.0 / (1.0 - 0.999 ** t)
        carried = lr * c1 * 4 * U32 * s_m / (np.sqrt(v * c2) + 1e-8)
        gates.check_abs(f"theta t={t}", p1 - th, 4 * U32 * np.abs(p0) + 16 * U32 * upd + carried, 1.0)
        gates.check(f"theta t={t}", p1, th, 1e-6, elementwise=False)
    gates.assert_all()


@pytest.mark.parametrize("wd", [0.0, 0.01])
def test_adamw_trajectory_matches_oracle(tmp_path, wd):
    """Five eager FP32 steps on changing batches and rates: the parameters after
    each step against the oracle's own five steps (its own FP64 gradients).  The
    FP32 gradients differ from the oracle's by < 1e-4, so each update differs by
    about that much relative; the gate on the accumulated change is 1e-3."""
    d, g, ctx, st, ost, delta, student = _setup(tmp_path, wd, 0)
    rng = np.random.default_rng(6)
    th = student.astype(np.float64).copy()
    m, v = np.zeros_like(th), np.zeros_like(th)
    gates = Gates(f"AdamW trajectory, wd = {wd}")
    for t in range(1, STEPS + 1):
        ids = rng.permutation(64)[:36 + 5 * t]
        lr = RATES[t - 1]
        b = ctx.collate(st, ids)
        ctx.forward(b, train=True)
        ctx.backward(b)
        ctx.step(lr)
        ob = oracle.collate(ost, ids, delta)
        _, grad, _, _ = oracle.backward(d, th, ob)
        oracle.adam(th, grad, m, v, t, lr=lr, wd=wd)
        p = ctx.get_params()
        gates.check(f"change t={t}", p.astype(np.float64) - student, th - student, 1e-3, elementwise=False)
        gates.check(f"theta t={t}", p, th, 1e-5, elementwise=False)
    ctx.check()
    gates.assert_all()
