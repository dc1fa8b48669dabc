"""MetaPath label index (TRW_PREP_LABEL_INDEX, GPU only).

The index is checked twice: its records against a stable partition of each
row by label computed here with numpy, and the walks that use it against the
oracle, which scans the labels of E_v at every step as Section 2.2 defines
the MetaPath Gather.  Walks must be bit-identical with and without the index."""
import time

import numpy as np
import pytest

import paper_2107_11983_gb300 as trw
import synth
from gpu_common import assert_paths_equal, oracle_alias, oracle_walk, rmat_graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def expected_index(g, stride):
    """Vertex records {v, g(v, 0..NL), padding = row end} and edge records =
    the vertex record of each destination in label-partitioned order."""
    nl = int(g.labels.max()) + 1 if g.ne else 1
    nv = g.nv
    vrec = np.zeros((nv, stride), dtype=np.int64)
    dst = np.empty(g.ne, dtype=np.int64)
    for v in range(nv):
        lo, hi = int(g.row_ptr[v]), int(g.row_ptr[v + 1])
        lab = g.labels[lo:hi]
        order = np.argsort(lab, kind="stable")
        counts = np.bincount(lab, minlength=nl)[:nl]
        starts = lo + np.concatenate([[0], np.cumsum(counts)])
        vrec[v, 0] = v
        vrec[v, 1:nl + 2] = starts
        vrec[v, nl + 2:] = hi
        dst[lo:hi] = g.col[lo:hi][order]
    return vrec.astype(np.int32), vrec[dst].astype(np.int32)


@pytest.mark.parametrize("nlabels,stride", [(5, 8), (6, 8), (7, 16), (14, 16), (15, 32), (30, 32)])
def test_index_records(nlabels, stride):
    g = rmat_graph(10, nlabels=nlabels)
    G = trw.Graph(g.row_ptr, g.col, None, g.labels)
    assert G.debug_label_index() is None
    G.prepare(trw.PREP_LABEL_INDEX)
    st, v, e = G.debug_label_index()
    assert st == stride
    ev, ee = expected_index(g, stride)
    assert np.array_equal(v, ev)
    assert np.array_equal(e, ee)
    G.prepare(trw.PREP_LABEL_INDEX)  # already built: nothing changes
    assert G.debug_label_index()[0] == stride


@pytest.mark.parametrize("nlabels", [5, 14, 30])
@pytest.mark.parametrize("kernel", [trw.KERNEL_PLAIN, trw.KERNEL_PERSISTENT], ids=["plain", "persistent"])
def test_indexed_metapath_matches_oracle(nlabels, kernel):
    g = rmat_graph(12, nlabels=nlabels)
    G = trw.Graph(g.row_ptr, g.col, None, g.labels)
    G.prepare(trw.PREP_LABEL_INDEX)
    src = np.concatenate([synth.vertex_sources(g.nv), synth.sources(1237, g.nv, seed=3)])
    for slen, seed in [(5, 1), (1, 2), (16, 3)]:
        schema = synth.schema(slen, nlabels, seed=seed)
        want = oracle_walk(g, trw.METAPATH, src, 80, seed=40 + seed, schema=schema)
        out = G.walk(trw.METAPATH, torch.from_numpy(src).cuda(), 80, seed=40 + seed, kernel=kernel, schema=schema)
        torch.cuda.synchronize()
        assert_paths_equal(out.paths.cpu().numpy(), out.lengths.cpu().numpy(), want)


def test_indexed_and_scanned_walks_identical():
    g = rmat_graph(12)
    schema = np.array([1, 3, 0, 4, 2], np.uint8)
    src = synth.sources(20000, g.nv, seed=8)
    scan = trw.Graph(g.row_ptr, g.col, None, g.labels)
    idx = trw.Graph(g.row_ptr, g.col, None, g.labels)
    idx.prepare(trw.PREP_LABEL_INDEX)
    a = scan.walk(trw.METAPATH, src, 60, seed=5, schema=schema, walks_per_source=3)
    b = idx.walk(trw.METAPATH, src, 60, seed=5, schema=schema, walks_per_source=3)
    assert np.array_equal(a.lengths, b.lengths)
    mask = np.arange(61)[None, :] < a.lengths[:, None]
    assert np.array_equal(a.paths[mask], b.paths[mask])


def test_indexed_mixed_batch_and_serve():
    g = rmat_graph(12)
    G = trw.Graph(g.row_ptr, g.col, g.weights, g.labels)
    G.prepare(trw.PREP_ALIAS | trw.PREP_LABEL_INDEX)
    reqs = [
        dict(algo=trw.PPR, sources=synth.sources(3000, g.nv, seed=4), max_len=1000, seed=21, ppr_stop=0.2,
             endpoints=True),
        dict(algo=trw.METAPATH, sources=synth.vertex_sources(g.nv), max_len=80, seed=22,
             schema=np.array([0, 1, 2, 3, 4], np.uint8)),
        dict(algo=trw.DEEPWALK_WEIGHTED, sources=synth.sources(777, g.nv, seed=5), max_len=40, seed=23),
        dict(algo=trw.METAPATH, sources=synth.sources(999, g.nv, seed=9), max_len=33, seed=24,
             schema=np.array([4, 4, 2], np.uint8), walks_per_source=3),
    ]

    def check(r, paths, lengths):
        kw = {k: r[k] for k in ("ppr_stop", "schema", "walks_per_source") if k in r}
        want = oracle_walk(g, r["algo"], r["sources"], r["max_len"], r["seed"],
                           alias=oracle_alias(12) if r["algo"] == trw.DEEPWALK_WEIGHTED else None,
                           endpoints_only=r.get("endpoints", False), **kw)
        assert_paths_equal(paths, lengths, want, endpoints=r.get("endpoints", False))

    outs = G.walk_batch(reqs)
    torch.cuda.synchronize()
    for r, o in zip(reqs, outs):
        check(r, o.paths.cpu().numpy(), o.lengths.cpu().numpy())

    S = trw.Server(G, max_requests=16)
    try:
        live = []
        for r in reqs:
            n = r["sources"].shape[0] * r.get("walks_per_source", 1)
            shape = (n,) if r.get("endpoints") else (n, r["max_len"] + 1)
            op = torch.full(shape, -1, dtype=torch.int32, device="cuda")
            ol = torch.full((n,), -1, dtype=torch.int32, device="cuda")
            kw = {k: r[k] for k in ("ppr_stop", "schema", "walks_per_source", "endpoints") if k in r}
            live.append((r, S.submit(r["algo"], r["sources"], r["max_len"], r["seed"], op, ol, **kw), op, ol))
        for r, rid, op, ol in live:
            t = time.time()
            while S.poll(rid) == trw.PENDING:
                assert time.time() - t < 60
                time.sleep(0.0005)
            check(r, op.cpu().numpy(), ol.cpu().numpy())
    finally:
        S.close()


def test_index_rejections():
    g = rmat_graph(10, nlabels=31)  # label 30 is one too many
    G = trw.Graph(g.row_ptr, g.col, None, g.labels)
    with pytest.raises(trw.TRWError) as e:
        G.prepare(trw.PREP_LABEL_INDEX)
    assert e.value.status == -1
    assert G.debug_label_index() is None
    # the scan still serves MetaPath on that graph
    src = synth.sources(500, g.nv, seed=1)
    schema = np.array([30, 0, 29], np.uint8)
    out = G.walk(trw.METAPATH, src, 20, seed=3, schema=schema)
    assert_paths_equal(out.paths, out.lengths, oracle_walk(g, trw.METAPATH, src, 20, seed=3, schema=schema))
    nol = trw.Graph(g.row_ptr, g.col, None, None)
    with pytest.raises(trw.TRWError) as e:
        nol.prepare(trw.PREP_LABEL_INDEX)
    assert e.value.status == -1
    with pytest.raises(trw.TRWError) as e:
        nol.prepare(64)
    assert e.value.status == -1


def test_index_degenerate_rows():
    # isolated vertices, a schema label no edge carries, one-edge rows
    g = synth.from_edges(6, [(0, 1), (1, 2), (2, 0), (2, 3), (3, 2)])
    g.labels = np.array([0, 1, 2, 2, 0], np.uint8)
    G = trw.Graph(g.row_ptr, g.col, None, g.labels)
    G.prepare(trw.PREP_LABEL_INDEX)
    st, v, e = G.debug_label_index()
    ev, ee = expected_index(g, st)
    assert np.array_equal(v, ev) and np.array_equal(e, ee)
    src = np.array([0, 1, 2, 3, 4, 5] * 40, np.int32)
    for schema in ([0, 1, 2], [2], [3], [2, 0], [2, 255, 0], [0, 6, 7, 8]):
        sch = np.array(schema, np.uint8)
        out = G.walk(trw.METAPATH, src, 12, seed=7, schema=sch)
        assert_paths_equal(out.paths, out.lengths, oracle_walk(g, trw.METAPATH, src, 12, seed=7, schema=sch))
