"""Continuous-batching inference server: each molecule's prediction is the same alone
and in any mix (bit-identical: row-invariant slots), matches the FP64 oracle, and the
queue admits by memory, validates requests and bounds its waits."""
import threading

import numpy as np
import pytest

import oracle
import synth
from gpu_common import context, write_both
from helpers import rel_norm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def model(tmp_path_factory):
    import paper_2207_11333_gb300 as g
    H, L = 32, 2
    gs = synth.molecules_uniform(41, 600, 5, 80)
    path, ost = write_both(gs, str(tmp_path_factory.mktemp("serve")))
    st = g.Store(path)
    delta = st.delta()
    ctx = context(H, L, 8, 2048, 8192, delta)
    p = synth.init_params(3, H, L)
    ctx.set_params(p)
    return g, gs, ost, delta, ctx, p, oracle.Dims(H=H, L=L)


@pytest.mark.parametrize("precision", [0, 1])
def test_alone_equals_mix_and_oracle(model, precision):
    g, gs, ost, delta, ctx, p, d = model
    srv = g.Server(ctx, n_slots=3, buckets=(512, 2048, 8192), max_graphs=300, precision=precision)
    alone = {}
    for i in range(0, 40, 4):                         # a few molecules, one request each
        t = srv.submit(*g.request_arrays(gs, i, 1))
        alone[i] = srv.wait(t)[0][0]
    # a burst of mixed requests submitted back to back (overlapping on the GPU)
    rng = np.random.default_rng(0)
    tickets = []
    pos = 0
    while pos < 600:
        n = int(min(600 - pos, rng.integers(1, 90)))
        tickets.append((pos, n, srv.submit(*g.request_arrays(gs, pos, n))))
        pos += n
    mix = np.zeros(600, np.float32)
    for first, n, t in tickets:
        out, lat = srv.wait(t)
        mix[first:first + n] = out
        assert lat > 0
    for i, v in alone.items():
        assert v == mix[i], (i, v, mix[i])          # bitwise: row-invariant arithmetic
    ob = oracle.collate(ost, np.arange(600), delta)
    ref = oracle.forward(d, p.astype(np.float64), ob)
    tol = 1e-5 if precision == 0 else 2e-2
    assert rel_norm(mix, ref) < tol, rel_norm(mix, ref)
    st = srv.stats()
    assert st["molecules"] == 600 + len(alone) and st["batches"] >= 2
    srv.close()


def test_admission_validation_and_timeouts(model):
    g, gs, ost, delta, ctx, p, d = model
    srv = g.Server(ctx, n_slots=1, buckets=(2048,), max_graphs=64, queue_nodes=3000)
    big = g.request_arrays(gs, 0, 60)                 # ~2500 atoms; the queue holds 3000
    admitted, refused = [], 0
    for _ in range(50):                               # a burst far above what one slot drains
        t = srv.submit(*big)
        if t is None:
            refused += 1
        else:
            admitted.append(t)
    assert refused >= 1 and srv.stats()["refused"] == refused
    for t in admitted:
        srv.wait(t)
    with pytest.raises(g.GcnnError, match="EINVAL"):  # an edge to a missing atom
        nn, ne, ty, ed = g.request_arrays(gs, 0, 1)
        ed = ed.copy()
        ed[0, 0] = 250
        srv.submit(nn, ne, ty, ed)
    with pytest.raises(g.GcnnError, match="EINVAL"):  # larger than the whole queue
        srv.submit(*g.request_arrays(gs, 0, 120))
    t = srv.submit(*g.request_arrays(gs, 0, 60))
    with pytest.raises(g.GcnnError, match="ETIMEDOUT"):
        srv.wait(t, timeout_s=0.0)
    srv.wait(t)
    srv.close()


def test_concurrent_submitters(model):
    g, gs, ost, delta, ctx, p, d = model
    srv = g.Server(ctx, n_slots=4, buckets=(1024, 4096), max_graphs=256)
    results = {}

    def client(k):
        first = 100 * k
        t = srv.submit(*g.request_arrays(gs, first, 100))
        results[k] = srv.wait(t)[0]

    threads = [threading.Thread(target=client, args=(k,)) for k in range(6)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    t = srv.submit(*g.request_arrays(gs, 0, 600))
    whole = srv.wait(t)[0]
    for k in range(6):
        assert np.array_equal(results[k], whole[100 * k:100 * k + 100])
    srv.close()


def test_request_pool_wraps_and_releases_in_order(model):
    """The device request pool is a ring: with room for 2,500 atoms and a
    stream of requests of up to ~1,500 atoms, rooms wrap around the end of the
    pool many times, batches stop where the pool wraps, and refused requests
    are admitted again once earlier ones are done and released.  Every
    prediction equals, bit for bit, that of a server whose pool never wraps."""
    g, gs, ost, delta, ctx, p, d = model
    small = g.Server(ctx, n_slots=2, buckets=(2048,), max_graphs=64, queue_nodes=2500)
    large = g.Server(ctx, n_slots=2, buckets=(2048,), max_graphs=64)
    rng = np.random.default_rng(7)
    spans, pos = [], 0
    for _ in range(40):
        n = int(rng.integers(3, 30))
        if pos + n > 600:
            pos = 0
        spans.append((pos, n))
        pos += n
    want = [large.wait(large.submit(*g.request_arrays(gs, a, n)))[0] for a, n in spans]
    outstanding, got, refusals, atoms = [], {}, 0, 0
    for k, (a, n) in enumerate(spans):
        req = g.request_arrays(gs, a, n)
        atoms += int(np.sum(req[0]))
        while True:
            t = small.submit(*req)
            if t is not None:
                outstanding.append((k, t))
                break
            refusals += 1
            k0, t0 = outstanding.pop(0)          # the oldest request frees its room first
            got[k0] = small.wait(t0)[0]
    for k0, t0 in outstanding:
        got[k0] = small.wait(t0)[0]
    assert atoms > 6 * 2500 and refusals > 0
    for k in range(len(spans)):
        assert np.array_equal(got[k], want[k]), k
    assert small.stats()["refused"] == refusals
    small.close()
    large.close()
