"""Largest and extreme arguments (GPU only), against the oracle: walk indices
that end exactly at 2^32, extreme seeds, long walks, the longest schema, a
batch of the maximum number of requests, and a hub row adjacent to almost
every vertex (every degree threshold of the kernels crossed at once)."""
import numpy as np
import pytest

import oracle
import paper_2107_11983_gb300 as trw
import synth
from gpu_common import assert_paths_equal, oracle_alias, oracle_walk, rmat_graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

KW = {
    trw.DEEPWALK: {},
    trw.DEEPWALK_WEIGHTED: {},
    trw.PPR: {"ppr_stop": 0.2},
    trw.NODE2VEC: {"n2v_p": 0.5, "n2v_q": 2.0},
    trw.METAPATH: {"schema": np.array([1, 3, 0, 4, 2], np.uint8)},
}


@pytest.fixture(scope="module")
def graph():
    g = rmat_graph(11)
    G = trw.Graph(g.row_ptr, g.col, g.weights, g.labels)
    G.prepare()
    return g, G


@pytest.mark.parametrize("algo", list(KW), ids=["deepwalk", "weighted", "ppr", "node2vec", "metapath"])
def test_walk_indices_end_at_2_pow_32(graph, algo):
    g, G = graph
    src = synth.sources(1000, g.nv, seed=2)
    off = 2 ** 32 - 3000  # walks off .. 2^32 - 1: the last counter value is used
    for seed in (0, 2 ** 64 - 1):
        want = oracle_walk(g, algo, src, 30, seed=seed, alias=oracle_alias(11) if algo == trw.DEEPWALK_WEIGHTED else None,
                           walks_per_source=3, walk_offset=off, **KW[algo])
        out = G.walk(algo, src, 30, seed=seed, walks_per_source=3, walk_offset=off, **KW[algo])
        assert_paths_equal(out.paths, out.lengths, want)
    with pytest.raises(trw.TRWError) as e:  # one walk past the counter range
        G.walk(algo, src, 30, seed=1, walks_per_source=3, walk_offset=off + 1, **KW[algo])
    assert e.value.status == -1


@pytest.mark.parametrize("algo", [trw.DEEPWALK_WEIGHTED, trw.NODE2VEC, trw.METAPATH], ids=["weighted", "node2vec", "metapath"])
def test_long_walks(graph, algo):
    g, G = graph
    src = synth.sources(200, g.nv, seed=5)
    want = oracle_walk(g, algo, src, 5000, seed=9, alias=oracle_alias(11) if algo == trw.DEEPWALK_WEIGHTED else None,
                       **KW[algo])
    for kernel in (trw.KERNEL_PLAIN, trw.KERNEL_PERSISTENT):
        out = G.walk(algo, src, 5000, seed=9, kernel=kernel, **KW[algo])
        assert_paths_equal(out.paths, out.lengths, want)


def test_longest_schema_and_largest_batch(graph):
    g, G = graph
    schema16 = synth.schema(16, 5, seed=3)
    out = G.walk(trw.METAPATH, synth.vertex_sources(g.nv), 80, seed=4, schema=schema16)
    assert_paths_equal(out.paths, out.lengths,
                       oracle_walk(g, trw.METAPATH, synth.vertex_sources(g.nv), 80, seed=4, schema=schema16))
    with pytest.raises((trw.TRWError, ValueError)):
        G.walk(trw.METAPATH, synth.vertex_sources(g.nv), 80, seed=4, schema=synth.schema(17, 5, seed=3))
    algos = list(KW)
    reqs = []
    for i in range(trw.MAX_BATCH):
        a = algos[i % len(algos)]
        reqs.append(dict(algo=a, sources=synth.sources(37 + 11 * i, g.nv, seed=100 + i), max_len=20 + i, seed=i,
                         **KW[a]))
    outs = G.walk_batch(reqs)
    torch.cuda.synchronize()
    for r, o in zip(reqs, outs):
        kw = {k: v for k, v in r.items() if k not in ("algo", "sources", "max_len", "seed")}
        want = oracle_walk(g, r["algo"], r["sources"], r["max_len"], r["seed"],
                           alias=oracle_alias(11) if r["algo"] == trw.DEEPWALK_WEIGHTED else None, **kw)
        assert_paths_equal(o.paths.cpu().numpy(), o.lengths.cpu().numpy(), want)
    with pytest.raises(ValueError):
        G.walk_batch(reqs + reqs[:1])


def test_hub_adjacent_to_almost_every_vertex():
    # a star of 200,000 leaves plus a sparse ring: the hub row crosses every
    # degree threshold (whole-block alias preparation, warp scans and
    # searches, the neighbour hash), and most walks pass through it
    n = 200_001
    leaves = np.arange(1, n, dtype=np.int64)
    ring = np.stack([leaves, np.roll(leaves, -1)], axis=1)
    edges = np.concatenate([np.stack([np.zeros(n - 1, np.int64), leaves], axis=1), ring[::3]])
    g = synth.from_edges(n, edges.tolist(), symmetric=True)
    g.weights = synth.edge_weights(g)
    g.labels = synth.edge_labels(g)
    src = np.concatenate([np.zeros(300, np.int32), synth.sources(3000, n, seed=6)])
    al = oracle.prepare_alias(g.row_ptr, g.weights)
    for prep in (trw.PREP_ALIAS, trw.PREP_ALL):
        G = trw.Graph(g.row_ptr, g.col, g.weights, g.labels)
        G.prepare(prep)
        for algo in KW:
            want = oracle_walk(g, algo, src, 40, seed=8, alias=al if algo == trw.DEEPWALK_WEIGHTED else None,
                               **KW[algo])
            out = G.walk(algo, src, 40, seed=8, **KW[algo])
            assert_paths_equal(out.paths, out.lengths, want)
