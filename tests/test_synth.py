"""The seeded input generator (CPU only): deterministic, valid CSR, attributes
keyed on the unordered endpoint pair."""
import numpy as np

import synth


def test_rmat_is_deterministic_across_thread_counts():
    a = synth.rmat(12, seed=3, nthreads=1)
    b = synth.rmat(12, seed=3, nthreads=7)
    assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col, b.col)
    c = synth.rmat(12, seed=4)
    assert not (a.ne == c.ne and np.array_equal(a.col, c.col))


def test_rmat_csr_valid_symmetric():
    g = synth.rmat(11, seed=2)
    assert g.row_ptr[0] == 0 and np.all(np.diff(g.row_ptr) >= 0) and g.row_ptr[-1] == g.ne
    edges = set()
    for v in range(g.nv):
        row = g.col[g.row_ptr[v]:g.row_ptr[v + 1]]
        assert np.all(np.diff(row) > 0), "sorted, no duplicates"
        assert not np.any(row == v), "no self-loops"
        assert np.all((row >= 0) & (row < g.nv))
        edges.update((v, int(c)) for c in row)
    assert all((b, a) in edges for a, b in edges), "symmetrised"
    assert g.ne <= 2 * 16 * g.nv
    d = g.degrees()
    assert d.max() > 20 * d.mean(), "power-law skew"


def test_rmat_directed_not_symmetric():
    g = synth.rmat(10, seed=2, symmetric=False)
    edges = {(v, int(c)) for v in range(g.nv) for c in g.col[g.row_ptr[v]:g.row_ptr[v + 1]]}
    assert any((b, a) not in edges for a, b in edges)


def test_weights_and_labels_keyed_on_pair():
    g = synth.rmat(10, seed=8)
    w = synth.edge_weights(g, seed=8)
    lab = synth.edge_labels(g, seed=8, nlabels=5)
    assert w.dtype == np.float32 and w.min() >= 1.0 and w.max() < 100.0
    assert lab.max() <= 4 and len(np.unique(lab)) == 5
    pos = {}
    for v in range(g.nv):
        for j in range(g.row_ptr[v], g.row_ptr[v + 1]):
            pos[(v, int(g.col[j]))] = j
    for (a, b), j in list(pos.items())[:5000]:
        k = pos[(b, a)]
        assert w[j] == w[k] and lab[j] == lab[k]


def test_sources_and_schema():
    s = synth.sources(100000, 12345, seed=1)
    assert s.min() >= 0 and s.max() < 12345
    assert np.array_equal(s, synth.sources(100000, 12345, seed=1))
    h = synth.schema(5, 5, seed=1)
    assert h.shape == (5,) and h.max() < 5
