"""Device collation against the oracle's collation: bit-exact integers and scalers."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import context, write_both

pytestmark = pytest.mark.gpu


def _compare(gb, ob):
    e = gb.export()
    assert np.array_equal(e["node_off"], ob.node_off.astype(np.int32))
    for k in ("graph_id", "row_ptr", "col", "rev", "deg", "types"):
        assert np.array_equal(e[k], getattr(ob, k)), k
    for k in ("amp", "att", "y"):
        assert np.array_equal(e[k].view(np.uint32), getattr(ob, k).view(np.uint32)), k


@pytest.mark.parametrize("resident", [False, True])
def test_collate_bit_exact(resident, tmp_path):
    import paper_2207_11333_gb300 as g
    gs = synth.molecules_uniform(1, 300, 1, 80)
    gs.y = synth.uniform_targets(9, 0, 300, 1, 10)
    path, ost = write_both(gs, str(tmp_path))
    st = g.Store(path)
    if resident:
        st.to_device()
    delta = st.delta()
    ctx = context(32, 1, 256, 256 * 80, 256 * 200, delta)
    rng = np.random.default_rng(3)
    cases = [rng.integers(0, 300, 200), np.arange(300)[:256][::-1], np.array([7]), rng.integers(0, 300, 33),
             np.array([0, 0, 0, 5, 5])]
    for ids in cases:
        gb = ctx.collate(st, ids)
        ob = oracle.collate(ost, ids, delta)
        assert (gb.n_graphs, gb.n_nodes, gb.n_edges) == (ob.G, ob.N, ob.E)
        _compare(gb, ob)
    ctx.check()


@pytest.mark.parametrize("resident", [False, True])
def test_collate_bit_exact_around_the_single_launch_limit(resident, tmp_path):
    """Batches of up to 1024 graphs are collated by one launch whose blocks each
    scan the whole batch's counts; larger ones by a scan launch and a per-graph
    launch.  Both sides of the limit, and a range of the device-resident order,
    match the oracle's collation bit for bit."""
    import paper_2207_11333_gb300 as g
    gs = synth.molecules_uniform(21, 3000, 1, 30)
    gs.y = synth.uniform_targets(22, 0, 3000, 1, 10)
    path, ost = write_both(gs, str(tmp_path))
    st = g.Store(path)
    if resident:
        st.to_device()
    delta = st.delta()
    ctx = context(32, 1, 2500, 2500 * 30, 2500 * 80, delta)
    rng = np.random.default_rng(23)
    for n in (1023, 1024, 1025, 2500):
        ids = rng.permutation(3000)[:n]
        gb = ctx.collate(st, ids)
        ob = oracle.collate(ost, ids, delta)
        assert (gb.n_graphs, gb.n_nodes, gb.n_edges) == (ob.G, ob.N, ob.E)
        _compare(gb, ob)
    if resident:
        order = rng.permutation(3000)
        ctx.set_order(st, order)
        for first, n in ((100, 1024), (400, 1800)):
            gb = ctx.collate_range(st, first, n)
            _compare(gb, oracle.collate(ost, order[first:first + n], delta))
    ctx.check()


def test_collate_edge_cases(tmp_path):
    import paper_2207_11333_gb300 as g
    from helpers import custom_set
    big = synth.make_graphs(4, np.array([255, 254, 3], np.int32))        # largest graphs the store allows
    tiny = custom_set([([2], []), ([0, 1], [(0, 1)])])                  # single atom (no edges), one bond
    gs = synth.GraphSet(np.concatenate([big.node_ptr, big.node_ptr[-1] + tiny.node_ptr[1:]]),
                        np.concatenate([big.edge_ptr, big.edge_ptr[-1] + tiny.edge_ptr[1:]]),
                        np.concatenate([big.types, tiny.types]), np.concatenate([big.edges, tiny.edges]),
                        np.arange(5, dtype=np.float32))
    path, ost = write_both(gs, str(tmp_path))
    st = g.Store(path)
    delta = st.delta()
    ctx = context(16, 1, 8, 1024, 4096, delta)
    for ids in ([0, 1, 2, 3, 4], [3], [4, 3], [1]):
        gb = ctx.collate(st, ids)
        _compare(gb, oracle.collate(ost, ids, delta))
    gb = ctx.collate(st, np.zeros(0, np.int64))                        # empty batch
    assert (gb.n_graphs, gb.n_nodes, gb.n_edges) == (0, 0, 0)
    with pytest.raises(g.GcnnError, match="capacity"):
        ctx.collate(st, [0, 1, 2, 0, 1, 0])                               # 1276 > 1024 nodes
    with pytest.raises(g.GcnnError, match="out of range"):
        ctx.collate(st, [9])
    ctx.check()


@pytest.mark.parametrize("F", [0, 4])
def test_collate_from_per_graph_files(tmp_path, F):
    """The per-graph-file loading path gives the batch of the packed store, bit-exact
    (bond features included) and equal to the oracle's collation."""
    import paper_2207_11333_gb300 as g
    gs = synth.molecules_uniform(11, 120, 3, 40)
    gs.y = synth.uniform_targets(12, 0, 120, 1, 10)
    if F:
        gs.eattr = synth.bond_features(13, gs, F)
    paths = synth.write_graph_files(str(tmp_path / "files"), gs)
    packed = str(tmp_path / "packed.gcnn")
    g.store_pack(paths, packed, 4)
    st = g.Store(packed)
    ost = oracle.read_store(packed)
    delta = st.delta()
    ctx = context(16, 1, 128, 128 * 40, 128 * 100, delta, F=F)
    ids = np.random.default_rng(5).integers(0, 120, 100)
    fb = ctx.collate_files([paths[i] for i in ids])
    fe = fb.export()
    fa = fb.tensor("edge_attr").cpu().numpy() if F else None
    sb = ctx.collate(st, ids)
    se = sb.export()
    for k in fe:
        assert np.array_equal(fe[k], se[k]), k
    if F:
        assert np.array_equal(fa, sb.tensor("edge_attr").cpu().numpy())
    _compare(sb, oracle.collate(ost, ids, delta))
    ctx.check()
