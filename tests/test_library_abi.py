"""The C-ABI library loads, exports every declared entry point, and its host-side
store reader agrees with the oracle (no GPU needed: no compute calls)."""
import os
import re

import numpy as np
import pytest

import oracle
import synth
from helpers import custom_set

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "gcnn.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gcnn_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported():
    import paper_2207_11333_gb300 as g
    names = _declared()
    assert len(names) >= 30
    missing = [n for n in names if not hasattr(g.lib, n)]
    assert not missing, missing


def test_version_and_error_text():
    import paper_2207_11333_gb300 as g
    assert g.lib.gcnn_version() >= 100
    assert isinstance(g.lib.gcnn_last_error(), bytes)


def test_store_reader_matches_oracle(tmp_path):
    import paper_2207_11333_gb300 as g
    gs = synth.molecules_uniform(1, 80, 3, 60)
    gs.y = synth.uniform_targets(5, 0, 80, 1, 10)
    path = str(tmp_path / "s.gcnn")
    synth.write_store(path, gs)
    st = g.Store(path)
    assert (st.n_graphs, st.n_nodes, st.n_edges) == (gs.n_graphs, gs.n_nodes, gs.n_edges)
    ost = oracle.read_store(path)
    assert st.delta() == oracle.delta_of(ost)            # same summation order: bitwise
    ids = np.array([5, 3, 3, 79, 0])
    assert st.batch_size(ids) == (int(np.sum(np.diff(gs.node_ptr)[ids])), int(np.sum(np.diff(gs.edge_ptr)[ids])))
    assert abs(st.delta(ids) - oracle.delta_of(ost, ids)) <= 1e-15 * st.delta(ids)


def _bad_store(tmp_path, gs, name):
    path = str(tmp_path / name)
    synth.write_store(path, gs)
    return path


def test_store_rejects_malformed_files(tmp_path):
    import paper_2207_11333_gb300 as g
    p = str(tmp_path / "junk")
    open(p, "wb").write(b"not a store at all" * 10)
    with pytest.raises(g.GcnnError, match="EFORMAT"):
        g.Store(p)
    # one direction of a bond missing
    gs = custom_set([([0, 1, 2], [(0, 1), (1, 2)])])
    gs.edges = gs.edges[:-1].copy()
    gs.edge_ptr = np.array([0, 3], np.int64)
    with pytest.raises(g.GcnnError, match="both directions"):
        g.Store(_bad_store(tmp_path, gs, "asym"))
    # atom type out of range
    gs = custom_set([([0, 9], [(0, 1)])])
    with pytest.raises(g.GcnnError, match="atom type"):
        g.Store(_bad_store(tmp_path, gs, "type"))
    # truncated file
    gs = synth.molecules_uniform(2, 4, 5, 9)
    path = _bad_store(tmp_path, gs, "trunc")
    data = open(path, "rb").read()
    open(path, "wb").write(data[:-70])
    with pytest.raises(g.GcnnError, match="EFORMAT"):
        g.Store(path)


def test_store_rejects_oversized_graph(tmp_path):
    import paper_2207_11333_gb300 as g
    gs = synth.make_graphs(3, np.array([10], np.int32))
    # claim 256 nodes for one graph
    gs.node_ptr = np.array([0, 256], np.int64)
    gs.types = np.zeros(256, np.uint8)
    with pytest.raises(g.GcnnError, match="nodes"):
        g.Store(_bad_store(tmp_path, gs, "big"))


def test_store_with_bond_features(tmp_path):
    """Version-2 stores: the feature count is read back; a bond whose two directions
    carry different features, or a feature count above 16, is rejected."""
    import paper_2207_11333_gb300 as g
    gs = synth.molecules_uniform(4, 10, 3, 20)
    gs.eattr = synth.bond_features(6, gs, 4)
    st = g.Store(_bad_store(tmp_path, gs, "bonds"))
    assert st.edge_features == 4 and st.n_edges == gs.n_edges
    assert g.Store(_bad_store(tmp_path, synth.molecules_uniform(4, 3, 3, 9), "plain")).edge_features == 0
    bad = gs.eattr.copy()
    bad[7, 2] += 1.0                     # one direction of one bond differs
    gs.eattr = bad
    with pytest.raises(g.GcnnError, match="differ in features"):
        g.Store(_bad_store(tmp_path, gs, "asym_feat"))
    gs.eattr = np.zeros((gs.n_edges, 17), np.float32)
    with pytest.raises(g.GcnnError, match="EFORMAT"):
        g.Store(_bad_store(tmp_path, gs, "too_many"))


@pytest.mark.parametrize("F", [0, 3])
def test_pack_per_graph_files_matches_store_writer(tmp_path, F):
    """gcnn_store_pack of one file per graph writes the same bytes as the store
    writer, whatever the thread count; a bad file is named in the error."""
    import paper_2207_11333_gb300 as g
    gs = synth.molecules_uniform(8, 40, 3, 30)
    gs.y = synth.uniform_targets(9, 0, 40, 1, 10)
    if F:
        gs.eattr = synth.bond_features(10, gs, F)
    paths = synth.write_graph_files(str(tmp_path / "files"), gs)
    ref = str(tmp_path / "ref.gcnn")
    synth.write_store(ref, gs)
    want = open(ref, "rb").read()
    for threads in (1, 3, 8):
        out = str(tmp_path / f"packed{threads}.gcnn")
        g.store_pack(paths, out, threads)
        assert open(out, "rb").read() == want
    st = g.Store(str(tmp_path / "packed8.gcnn"))
    assert (st.n_graphs, st.edge_features) == (40, F)
    bad = open(paths[7], "rb").read()
    open(paths[7], "wb").write(bad[:-1])
    with pytest.raises(g.GcnnError, match="g0000007"):
        g.store_pack(paths, str(tmp_path / "x.gcnn"), 4)


def test_store_with_node_targets(tmp_path):
    """Version-2 stores may carry node-level targets (with or without bond features);
    the library reports them and the oracle reads them back."""
    import paper_2207_11333_gb300 as g
    gs = synth.molecules_uniform(12, 9, 3, 20)
    gs.ynode = synth.uniform(13, 0, gs.n_nodes, -1.0, 1.0).astype(np.float32)
    for F in (0, 2):
        gs.eattr = synth.bond_features(14, gs, F) if F else None
        path = _bad_store(tmp_path, gs, f"ynode{F}")
        st = g.Store(path)
        assert st.has_node_targets and st.edge_features == F
        ost = oracle.read_store(path)
        assert np.array_equal(ost.ynode, gs.ynode)
    assert not g.Store(_bad_store(tmp_path, synth.molecules_uniform(12, 3, 3, 9), "plain2")).has_node_targets
