"""The seeded generators: determinism, graph invariants, distribution targets (no GPU)."""
import numpy as np

import synth


def test_streams_are_deterministic_and_distinct():
    a = synth.lib().synth_stream_first(1, 0, 0)
    assert a == synth.lib().synth_stream_first(1, 0, 0)
    assert len({synth.lib().synth_stream_first(s, g, p) for s in (1, 2) for g in range(50) for p in range(4)}) == 400


def test_molecule_graph_invariants():
    gs = synth.molecules_uniform(1, 200, 3, 80)
    assert gs.edges.shape[1] == 2
    for g in range(gs.n_graphs):
        n = int(gs.node_ptr[g + 1] - gs.node_ptr[g])
        e = gs.edges[gs.edge_ptr[g]:gs.edge_ptr[g + 1]].astype(np.int64)
        assert np.all(e < n) and np.all(e[:, 0] != e[:, 1])
        pairs = set(map(tuple, e.tolist()))
        assert len(pairs) == len(e), "multi-edge"
        assert all((v, u) in pairs for u, v in pairs), "not symmetric"
        deg = np.bincount(e[:, 1], minlength=n)
        assert deg.max() <= 4
        # connected: a spanning tree is always present
        seen, stack = {0}, [0]
        adj = [[] for _ in range(n)]
        for u, v in e:
            adj[u].append(v)
        while stack:
            u = stack.pop()
            for v in adj[u]:
                if v not in seen:
                    seen.add(v)
                    stack.append(v)
        assert len(seen) == n


def test_lognormal_counts_mean_and_range():
    gs = synth.molecules_lognormal(10, 20000)
    n = np.diff(gs.node_ptr)
    assert n.min() >= 3 and n.max() <= 51
    assert abs(n.mean() - 18.0) < 0.15
    assert abs(gs.n_edges / gs.n_nodes - 2.2) < 0.05


def test_type_frequencies():
    gs = synth.molecules_uniform(1, 3000, 5, 30)
    f = np.bincount(gs.types, minlength=7) / gs.n_nodes
    assert np.allclose(f, [.45, .33, .08, .08, .02, .02, .02], atol=0.01)


def test_regenerating_a_subset_matches():
    full = synth.molecules_uniform(7, 50, 5, 30)
    part = synth.make_graphs(7, synth.node_counts_uniform(7, 20, 10, 5, 30), g0=20)
    sub = full.subset(np.arange(20, 30))
    assert np.array_equal(part.node_ptr, sub.node_ptr) and np.array_equal(part.edges, sub.edges)
    assert np.array_equal(part.types, sub.types)


def test_param_init_ranges():
    H, L = 16, 2
    p = synth.init_params(3, H, L)
    assert p.size == synth.param_count(H, L)
    emb = p[:7 * H]
    assert abs(emb.mean()) < 0.3 and 0.6 < emb.std() < 1.4
    msg_w = p[7 * H:7 * H + 2 * H * H]
    assert np.abs(msg_w).max() <= 1 / np.sqrt(2 * H)


def test_store_version2_round_trip_with_bond_features(tmp_path):
    """A set with bond features is written as a version-2 store and read back unchanged;
    both directions of a bond carry the same features."""
    import oracle
    gs = synth.molecules_uniform(3, 12, 3, 20)
    gs.y = synth.uniform_targets(4, 0, 12, 1, 10)
    gs.eattr = synth.bond_features(5, gs, 3)
    assert gs.eattr.shape == (gs.n_edges, 3)
    assert np.array_equal(gs.eattr[0::2], gs.eattr[1::2])
    path = str(tmp_path / "b.gcnn")
    synth.write_store(path, gs)
    raw = np.fromfile(path, np.uint8)
    assert raw[8:12].view("<u4")[0] == 2
    st = oracle.read_store(path)
    assert st.F == 3
    assert np.array_equal(st.eattr, gs.eattr)
    assert np.array_equal(st.edges, gs.edges.reshape(-1)) and np.array_equal(st.y, gs.y)
    sub = gs.subset([5, 2])
    assert np.array_equal(sub.eattr, np.concatenate([gs.eattr[gs.edge_ptr[5]:gs.edge_ptr[6]],
                                                     gs.eattr[gs.edge_ptr[2]:gs.edge_ptr[3]]]))
