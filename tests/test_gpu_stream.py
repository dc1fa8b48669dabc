"""Streaming output (trw_walk_stream, trw_walk_to_file; GPU only): the slices
handed to the consumer, and the files written, hold the oracle's walks in
walk order; a consumer can stop the stream; invalid calls deliver nothing."""
import numpy as np
import pytest

import paper_2107_11983_gb300 as trw
import synth
from gpu_common import oracle_alias, oracle_walk, rmat_graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = {
    "weighted": (trw.DEEPWALK_WEIGHTED, 40, {}),
    "node2vec": (trw.NODE2VEC, 30, {"n2v_p": 0.5, "n2v_q": 2.0}),
    "ppr": (trw.PPR, 200, {"ppr_stop": 0.2}),
}


@pytest.fixture(scope="module")
def graph():
    g = rmat_graph(12)
    G = trw.Graph(g.row_ptr, g.col, g.weights, g.labels)
    G.prepare(trw.PREP_ALIAS)
    return g, G


def oracle_of(g, algo, src, L, seed, kw, **extra):
    return oracle_walk(g, algo, src, L, seed, alias=oracle_alias(12) if algo == trw.DEEPWALK_WEIGHTED else None,
                       **kw, **extra)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("device_sources", [False, True], ids=["host-src", "device-src"])
def test_stream_slices_match_oracle(graph, case, device_sources):
    g, G = graph
    algo, L, kw = CASES[case]
    src = synth.sources(5000, g.nv, seed=3)
    want = oracle_of(g, algo, src, L, 11, kw, walks_per_source=3)
    got_p, got_l, firsts = [], [], []

    def consume(first, paths, lengths):
        firsts.append((first, lengths.shape[0]))
        got_p.append(paths.copy())
        got_l.append(lengths.copy())

    s = torch.from_numpy(src).cuda() if device_sources else src
    moves = G.walk_stream(algo, s, L, 11, consume, slice_walks=1000, walks_per_source=3, **kw)
    # slices of 333 sources (999 walks), in order
    assert [f for f, _ in firsts] == list(range(0, 15000, 999))
    assert all(n == 999 for _, n in firsts[:-1]) and sum(n for _, n in firsts) == 15000
    lens = np.concatenate(got_l)
    paths = np.concatenate(got_p)
    assert np.array_equal(lens, want.lengths)
    mask = np.arange(L + 1)[None, :] < lens[:, None]
    assert np.array_equal(paths[mask], want.paths[mask])
    assert moves == want.stats["moves"]


def test_stream_endpoints_and_files(graph, tmp_path):
    g, G = graph
    src = synth.sources(3000, g.nv, seed=5)
    algo, L, kw = CASES["ppr"]
    ends = oracle_of(g, algo, src, L, 2, kw, endpoints_only=True)
    got = []
    G.walk_stream(algo, src, L, 2, lambda f, p, l: got.append(p.copy()), slice_walks=700, endpoints=True, **kw)
    assert np.array_equal(np.concatenate(got), ends.paths)
    for case in ("weighted", "node2vec"):
        algo, L, kw = CASES[case]
        want = oracle_of(g, algo, src, L, 9, kw)
        pf, lf = tmp_path / f"{case}.paths", tmp_path / f"{case}.len"
        moves = G.walk_to_file(algo, src, L, 9, str(pf), str(lf), **kw)
        lens = np.fromfile(lf, dtype=np.int32)
        flat = np.fromfile(pf, dtype=np.int32)
        assert np.array_equal(lens, want.lengths) and moves == want.stats["moves"]
        mask = np.arange(L + 1)[None, :] < want.lengths[:, None]
        assert np.array_equal(flat, want.paths[mask])  # row-major: walk after walk, no padding
    pf, lf = tmp_path / "ends.paths", tmp_path / "ends.len"
    G.walk_to_file(trw.PPR, src, 200, 2, str(pf), str(lf), endpoints=True, ppr_stop=0.2)
    assert np.array_equal(np.fromfile(pf, dtype=np.int32), ends.paths)


def test_stream_tiny_slices(graph):
    # slice_walks below walks_per_source: one source per slice
    g, G = graph
    src = synth.sources(40, g.nv, seed=12)
    algo, L, kw = CASES["node2vec"]
    want = oracle_of(g, algo, src, L, 4, kw, walks_per_source=5)
    firsts, got_l = [], []
    G.walk_stream(algo, src, L, 4, lambda f, p, ln: (firsts.append(f), got_l.append(ln.copy())) and None,
                  slice_walks=2, walks_per_source=5, **kw)
    assert firsts == list(range(0, 200, 5))
    assert np.array_equal(np.concatenate(got_l), want.lengths)


def test_stream_stop_errors_and_exceptions(graph, tmp_path):
    g, G = graph
    src = synth.sources(4000, g.nv, seed=6)
    seen = []

    def stop_after_two(first, paths, lengths):
        seen.append(first)
        return len(seen) == 2

    with pytest.raises(trw.TRWError) as e:
        G.walk_stream(trw.DEEPWALK, src, 20, 1, stop_after_two, slice_walks=500)
    assert e.value.status == trw.ERR_STOPPED and seen == [0, 500]

    def boom(first, paths, lengths):
        raise KeyError("consumer failed")

    with pytest.raises(KeyError):
        G.walk_stream(trw.DEEPWALK, src, 20, 1, boom, slice_walks=500)
    called = []
    bad = src.copy()
    bad[3000] = g.nv + 1
    with pytest.raises(trw.TRWError) as e:
        G.walk_stream(trw.DEEPWALK, bad, 20, 1, lambda *a: called.append(1), slice_walks=500)
    assert e.value.status == -1 and not called
    with pytest.raises(trw.TRWError) as e:
        G.walk_stream(trw.DEEPWALK, torch.from_numpy(bad).cuda(), 20, 1, lambda *a: called.append(1), slice_walks=500)
    assert e.value.status == -1 and not called
    with pytest.raises(trw.TRWError) as e:
        G.walk_to_file(trw.DEEPWALK, src, 20, 1, str(tmp_path / "no" / "such" / "dir"), str(tmp_path / "l"))
    assert e.value.status == trw.ERR_IO
    # the graph still walks after every failure
    out = G.walk(trw.DEEPWALK, src[:10], 5, seed=1)
    assert np.array_equal(out.lengths, oracle_of(g, trw.DEEPWALK, src[:10], 5, 1, {}).lengths)
