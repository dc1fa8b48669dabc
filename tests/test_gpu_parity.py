"""CUDA path against the oracle, element by element (GPU only).

Walks are bit-exact: every path vertex and length must equal the oracle's,
for every algorithm, for both kernels, for host and device buffers, at sizes
that span many warps and chunks with ragged tails."""
import numpy as np
import pytest

import oracle
import paper_2107_11983_gb300 as trw
import synth
from gpu_common import assert_paths_equal, oracle_alias, oracle_walk, rmat_graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SCALE = 12
ALGO_KW = {
    trw.DEEPWALK: {},
    trw.DEEPWALK_WEIGHTED: {},
    trw.PPR: {"ppr_stop": 0.2},
    trw.NODE2VEC: {"n2v_p": 0.5, "n2v_q": 2.0},
    trw.METAPATH: {"schema": np.array([1, 3, 0, 4, 2], np.uint8)},
}


@pytest.fixture(scope="module")
def small():
    g = rmat_graph(SCALE)
    G = trw.Graph(g.row_ptr, g.col, g.weights, g.labels)
    G.prepare()
    return g, G


def test_device_philox_matches_oracle():
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 2 ** 32, size=(257, 4), dtype=np.uint64).astype(np.uint32)
    for key in [(0, 0), (0xFFFFFFFF, 0xFFFFFFFF), (0xA4093822, 0x299F31D0), (1, 0)]:
        dev = trw.philox_device(ctr, *key)
        for i in range(ctr.shape[0]):
            assert np.array_equal(dev[i], oracle.philox4x32_10(ctr[i], key)), (i, key)


def test_alias_tables_match_oracle(small):
    g, G = small
    al = oracle_alias(SCALE)
    H, first, second = G.debug_alias()
    ne = g.ne
    Ho = al.H
    full = Ho == (1 << 32)
    assert np.array_equal(H[~full], Ho[~full].astype(np.uint32))
    assert np.all(H[full] == 0xFFFFFFFF)
    off = np.repeat(g.row_ptr[:-1], np.diff(g.row_ptr))
    assert np.array_equal(first, g.col[off + al.A_first])
    sec_slot = np.where(al.A_second >= 0, al.A_second, al.A_first)
    assert np.array_equal(second, g.col[off + sec_slot])
    assert ne == H.shape[0]


def _rows_graph(degrees, seed=11):
    """Directed CSR graph whose rows have the given degrees (random sorted
    distinct neighbours), with a different weight pattern per row."""
    rng = np.random.default_rng(seed)
    nv = max(max(degrees) + 1, len(degrees))
    row_ptr = np.zeros(nv + 1, dtype=np.int64)
    cols, ws = [], []
    for v in range(nv):
        d = degrees[v] if v < len(degrees) else int(rng.integers(0, 9))
        c = np.sort(rng.choice(nv, size=d, replace=False)).astype(np.int32)
        kind = v % 7
        if kind == 0:
            w = rng.uniform(1, 100, d)
        elif kind == 1:
            w = np.full(d, 3.0)
        elif kind == 2:  # one heavy edge absorbs every small one
            w = np.ones(d)
            if d:
                w[rng.integers(d)] = 1e4
        elif kind == 3:  # heavy-tailed: larges turn small again and again
            w = rng.geometric(0.3, d).astype(np.float64) ** 3
        elif kind == 4:  # half zeros
            w = rng.uniform(0, 1, d) * (rng.uniform(0, 1, d) < 0.5)
        elif kind == 5:
            w = np.where(np.arange(d) % 7 == 0, 1000.0, 1.0)
        else:  # quantisation extremes, S above 2^32
            w = rng.choice([1e-6, 0.5, 65535.0, 2.0], d)
        row_ptr[v + 1] = row_ptr[v] + d
        cols.append(c)
        ws.append(w.astype(np.float32))
    return synth.Graph(row_ptr, np.concatenate(cols), np.concatenate(ws))


def test_alias_tables_long_rows_match_oracle():
    # Rows on both sides of the whole-block threshold (4096 edges) and far
    # above it, each weight pattern at several lengths.
    degrees = [20000, 4095, 4096, 4097, 9001, 12000, 6000, 40000, 4096, 5000, 8191, 8192, 30000, 4100, 0, 1, 31, 32,
               33, 1000]
    g = _rows_graph(degrees)
    G = trw.Graph(g.row_ptr, g.col, g.weights, None)
    G.prepare()
    al = oracle.prepare_alias(g.row_ptr, g.weights)
    H, first, second = G.debug_alias()
    full = al.H == (1 << 32)
    assert np.array_equal(H[~full], al.H[~full].astype(np.uint32))
    assert np.all(H[full] == 0xFFFFFFFF)
    off = np.repeat(g.row_ptr[:-1], np.diff(g.row_ptr))
    live = ~np.repeat(al.dead.astype(bool), np.diff(g.row_ptr))
    assert np.array_equal(first[live], g.col[off + al.A_first][live])
    sec_slot = np.where(al.A_second >= 0, al.A_second, al.A_first)
    assert np.array_equal(second[live], g.col[off + sec_slot][live])
    assert np.all(first[~live] == -1) and np.all(second[~live] == -1)
    # and the walks over them
    src = np.concatenate([np.arange(len(degrees), dtype=np.int32), synth.sources(3001, g.nv, seed=4)])
    out = G.walk(trw.DEEPWALK_WEIGHTED, src, 40, seed=9)
    want = oracle.walk(g.row_ptr, g.col, oracle.DEEPWALK_WEIGHTED, src, 40, 9, alias=al)
    assert_paths_equal(out.paths, out.lengths, want)


def test_alias_dead_and_zero_weights():
    # vertex 0: all zero weights (dead for weighted walks); vertex 1: one zero weight
    g = synth.from_edges(4, [(0, 1), (0, 2), (1, 0), (1, 2), (1, 3), (2, 3), (3, 0)])
    w = np.array([0.0, 0.0, 0.0, 2.5, 1.0, 7.0, 3.0], dtype=np.float32)
    G = trw.Graph(g.row_ptr, g.col, w, None)
    G.prepare()
    al = oracle.prepare_alias(g.row_ptr, w)
    assert list(al.dead) == [1, 0, 0, 0]
    src = np.array([0, 1, 2, 3] * 50, np.int32)
    out = G.walk(trw.DEEPWALK_WEIGHTED, src, 6, seed=5)
    want = oracle.walk(g.row_ptr, g.col, oracle.DEEPWALK_WEIGHTED, src, 6, 5, alias=al)
    assert_paths_equal(out.paths, out.lengths, want)


@pytest.mark.parametrize("kernel", [trw.KERNEL_PLAIN, trw.KERNEL_PERSISTENT], ids=["plain", "persistent"])
@pytest.mark.parametrize("algo", list(ALGO_KW), ids=lambda a: ["deepwalk", "weighted", "ppr", "node2vec", "metapath"][a])
def test_walk_parity_device_buffers(small, algo, kernel):
    g, G = small
    # every vertex once plus a ragged tail of random sources
    src = np.concatenate([synth.vertex_sources(g.nv), synth.sources(1237, g.nv, seed=3)])
    L = 80 if algo != trw.PPR else 200
    want = oracle_walk(g, algo, src, L, seed=7, alias=oracle_alias(SCALE) if algo == trw.DEEPWALK_WEIGHTED else None,
                       **ALGO_KW[algo])
    out = G.walk(algo, torch.from_numpy(src).cuda(), L, seed=7, kernel=kernel, **ALGO_KW[algo])
    torch.cuda.synchronize()
    assert_paths_equal(out.paths.cpu().numpy(), out.lengths.cpu().numpy(), want)
    assert G.last_stats()["moves"] == int((want.lengths - 1).sum())


@pytest.mark.parametrize("algo", list(ALGO_KW), ids=lambda a: ["deepwalk", "weighted", "ppr", "node2vec", "metapath"][a])
def test_walk_parity_host_buffers_and_options(small, algo):
    g, G = small
    src = synth.sources(999, g.nv, seed=11)
    al = oracle_alias(SCALE) if algo == trw.DEEPWALK_WEIGHTED else None
    # several walks per source, a walk offset, host numpy buffers
    want = oracle_walk(g, algo, src, 33, seed=2 ** 40 + 3, alias=al, walks_per_source=3, walk_offset=12345,
                       **ALGO_KW[algo])
    out = G.walk(algo, src, 33, seed=2 ** 40 + 3, walks_per_source=3, walk_offset=12345, **ALGO_KW[algo])
    assert_paths_equal(out.paths, out.lengths, want)
    # endpoints only
    want = oracle_walk(g, algo, src, 50, seed=9, alias=al, endpoints_only=True, **ALGO_KW[algo])
    out = G.walk(algo, src, 50, seed=9, endpoints=True, **ALGO_KW[algo])
    assert_paths_equal(out.paths, out.lengths, want, endpoints=True)


def test_edge_cases(small):
    g, G = small
    src = synth.vertex_sources(g.nv)
    # max_len 0: every walk is its source
    out = G.walk(trw.DEEPWALK, src, 0, seed=1)
    assert np.all(out.lengths == 1) and np.array_equal(out.paths[:, 0], src)
    # empty batch
    out = G.walk(trw.NODE2VEC, np.zeros(0, np.int32), 10, seed=1, n2v_p=0.5, n2v_q=2.0)
    assert out.lengths.shape == (0,)
    # isolated vertices stop at once
    iso = np.nonzero(np.diff(g.row_ptr) == 0)[0].astype(np.int32)
    assert iso.size > 0
    out = G.walk(trw.DEEPWALK, iso, 10, seed=1)
    assert np.all(out.lengths == 1)
    # PPR stop 1: stop before the first move; stop 0: the whole length
    out = G.walk(trw.PPR, src, 10, seed=1, ppr_stop=1.0)
    assert np.all(out.lengths == 1)
    want = oracle_walk(g, trw.DEEPWALK, src, 10, seed=1)
    out = G.walk(trw.PPR, src, 10, seed=1, ppr_stop=0.0)
    assert_paths_equal(out.paths, out.lengths, want)


def test_invalid_arguments_write_nothing(small):
    g, G = small
    L = 5
    sentinel = -7
    bad = np.array([0, 1, g.nv], np.int32)
    paths = np.full((3, L + 1), sentinel, np.int32)
    lens = np.full(3, sentinel, np.int32)
    with pytest.raises(trw.TRWError) as e:
        G.walk(trw.DEEPWALK, bad, L, seed=1, out_paths=paths, out_lengths=lens)
    assert e.value.status == -1
    assert np.all(paths == sentinel) and np.all(lens == sentinel)
    # device sources out of range: rejected on the device before any write
    dsrc = torch.tensor([0, -1, 2], dtype=torch.int32, device="cuda")
    dp = torch.full((3, L + 1), sentinel, dtype=torch.int32, device="cuda")
    dl = torch.full((3,), sentinel, dtype=torch.int32, device="cuda")
    with pytest.raises(trw.TRWError) as e:
        G.walk(trw.DEEPWALK, dsrc, L, seed=1, out_paths=dp, out_lengths=dl)
    assert e.value.status == -1
    assert bool((dp == sentinel).all()) and bool((dl == sentinel).all())
    # device sources, host outputs: still nothing written
    hp = np.full((3, L + 1), sentinel, np.int32)
    hl = np.full(3, sentinel, np.int32)
    with pytest.raises(trw.TRWError) as e:
        G.walk(trw.DEEPWALK, dsrc, L, seed=1, out_paths=hp, out_lengths=hl)
    assert e.value.status == -1
    assert np.all(hp == sentinel) and np.all(hl == sentinel)
    src = np.array([0], np.int32)
    for kw in [dict(algo=trw.NODE2VEC, n2v_p=0.0), dict(algo=trw.NODE2VEC, n2v_q=-1.0),
               dict(algo=trw.PPR, ppr_stop=1.5), dict(algo=trw.METAPATH, schema=np.zeros(17, np.uint8)),
               dict(algo=trw.METAPATH, schema=None)]:
        algo = kw.pop("algo")
        with pytest.raises(trw.TRWError) as e:
            G.walk(algo, src, L, seed=1, **kw)
        assert e.value.status == -1, kw
    with pytest.raises(trw.TRWError):
        G.walk(trw.DEEPWALK, src, -1, seed=1)
    # a graph without weights cannot run weighted walks; without prepare: NOT_PREPARED
    G2 = trw.Graph(g.row_ptr, g.col, g.weights, None)
    with pytest.raises(trw.TRWError) as e:
        G2.walk(trw.DEEPWALK_WEIGHTED, src, L, seed=1)
    assert e.value.status == -3
    with pytest.raises(trw.TRWError) as e:
        G2.walk(trw.METAPATH, src, L, seed=1, schema=[0])
    assert e.value.status == -1
    # unsorted rows: node2vec refused, other walks fine
    rp = np.array([0, 2, 3, 4], np.int64)
    col = np.array([2, 1, 0, 0], np.int32)
    G3 = trw.Graph(rp, col)
    with pytest.raises(trw.TRWError) as e:
        G3.walk(trw.NODE2VEC, np.array([0], np.int32), 3, seed=1, n2v_p=0.5, n2v_q=2.0)
    assert e.value.status == -1
    G3.walk(trw.DEEPWALK, np.array([0], np.int32), 3, seed=1)
    # column id out of range is refused at load
    with pytest.raises(trw.TRWError):
        trw.Graph(np.array([0, 1], np.int64), np.array([5], np.int32))
    with pytest.raises(trw.TRWError):
        trw.Graph(np.array([0, 2, 1], np.int64), np.array([1, 0], np.int32))


def test_bad_weight_refused_at_load():
    g = synth.from_edges(3, [(0, 1), (1, 2), (2, 0)])
    for bad in (-2.0, float("nan"), float("inf"), -0.0001):
        with pytest.raises(trw.TRWError) as e:
            trw.Graph(g.row_ptr, g.col, np.array([1.0, bad, 1.0], np.float32))
        assert e.value.status == -1
    with pytest.raises(ValueError):
        trw.Graph(g.row_ptr, g.col, np.array([1.0, 1.0], np.float32))
    G = trw.Graph(g.row_ptr, g.col, np.array([1.0, 0.0, 1e30], np.float32))  # zero and huge weights are valid
    G.prepare(trw.PREP_ALL & ~trw.PREP_LABEL_INDEX)


def test_mixed_batch_one_launch(small):
    g, G = small
    al = oracle_alias(SCALE)
    reqs = [
        dict(algo=trw.PPR, sources=synth.sources(3000, g.nv, seed=4), max_len=1000, seed=21, ppr_stop=0.2,
             endpoints=True),
        dict(algo=trw.METAPATH, sources=synth.vertex_sources(g.nv), max_len=80, seed=22,
             schema=np.array([0, 1, 2, 3, 4], np.uint8)),
        dict(algo=trw.DEEPWALK_WEIGHTED, sources=synth.sources(777, g.nv, seed=5), max_len=40, seed=23),
        dict(algo=trw.NODE2VEC, sources=synth.sources(555, g.nv, seed=6), max_len=30, seed=24, n2v_p=0.5, n2v_q=2.0),
        dict(algo=trw.DEEPWALK, sources=synth.sources(1, g.nv, seed=7), max_len=80, seed=25, walks_per_source=100),
    ]
    outs = G.walk_batch(reqs)
    torch.cuda.synchronize()
    for r, o in zip(reqs, outs):
        kw = {k: r[k] for k in ("ppr_stop", "schema") if k in r}
        if r["algo"] == trw.NODE2VEC:
            kw.update(n2v_p=r["n2v_p"], n2v_q=r["n2v_q"])
        want = oracle_walk(g, r["algo"], r["sources"], r["max_len"], r["seed"],
                           alias=al if r["algo"] == trw.DEEPWALK_WEIGHTED else None,
                           endpoints_only=r.get("endpoints", False), walks_per_source=r.get("walks_per_source", 1),
                           **kw)
        assert_paths_equal(o.paths.cpu().numpy(), o.lengths.cpu().numpy(), want, endpoints=r.get("endpoints", False))


def test_sliced_host_outputs_large_batch():
    """A batch large enough to walk in slices (copy-out overlapped with the next
    slice) gives the oracle's paths, with several walks per source and an offset."""
    g = rmat_graph(14)
    G = trw.Graph(g.row_ptr, g.col, g.weights, g.labels)
    G.prepare()
    src = synth.sources(300_001, g.nv, seed=21)
    al = oracle.prepare_alias(g.row_ptr, g.weights)
    for algo, kw in [(trw.DEEPWALK_WEIGHTED, {}), (trw.NODE2VEC, {"n2v_p": 0.5, "n2v_q": 2.0})]:
        want = oracle_walk(g, algo, src, 20, seed=23, alias=al if algo == trw.DEEPWALK_WEIGHTED else None,
                           walks_per_source=4, walk_offset=77, **kw)
        h_paths = torch.full((src.shape[0] * 4, 21), -1, dtype=torch.int32).pin_memory()
        h_len = torch.full((src.shape[0] * 4,), -1, dtype=torch.int32).pin_memory()
        G.walk(algo, src, 20, seed=23, walks_per_source=4, walk_offset=77, out_paths=h_paths.numpy(),
               out_lengths=h_len.numpy(), **kw)
        assert_paths_equal(h_paths.numpy(), h_len.numpy(), want)
        assert G.last_stats()["moves"] == int((want.lengths - 1).sum())


def test_results_independent_of_tuning(small):
    g, G = small
    src = synth.vertex_sources(g.nv)
    kw = ALGO_KW[trw.NODE2VEC]
    want = oracle_walk(g, trw.NODE2VEC, src, 40, seed=3, **kw)
    old = G.tuning()
    try:
        for bt, ch, cd, sd in [(128, 1, 8, 33), (512, 7, 100000, 0x7fffffff), (64, 128, 32, 100), (96, 3, 1, 40)]:
            G.set_tuning(block_threads=bt, chunk=ch, coop_degree=cd, search_degree=sd, blocks_per_sm=1)
            out = G.walk(trw.NODE2VEC, src, 40, seed=3, **kw)
            assert_paths_equal(out.paths, out.lengths, want)
    finally:
        G.set_tuning(**old)


def test_autotune_keeps_results(small):
    g, G = small
    src = synth.vertex_sources(g.nv)
    want = oracle_walk(g, trw.METAPATH, src, 20, seed=4, schema=ALGO_KW[trw.METAPATH]["schema"])
    best = G.autotune(trw.METAPATH, 10, schema=ALGO_KW[trw.METAPATH]["schema"])
    assert best["block_threads"] in (64, 128, 256, 512)
    out = G.walk(trw.METAPATH, src, 20, seed=4, schema=ALGO_KW[trw.METAPATH]["schema"])
    assert_paths_equal(out.paths, out.lengths, want)


def test_directed_graph_parity():
    g = rmat_graph(11, seed=9, symmetric=False)
    G = trw.Graph(g.row_ptr, g.col, g.weights, g.labels)
    G.prepare()
    al = oracle.prepare_alias(g.row_ptr, g.weights)
    src = synth.vertex_sources(g.nv)
    for algo in ALGO_KW:
        want = oracle_walk(g, algo, src, 25, seed=31, alias=al if algo == trw.DEEPWALK_WEIGHTED else None,
                           **ALGO_KW[algo])
        out = G.walk(algo, src, 25, seed=31, **ALGO_KW[algo])
        assert_paths_equal(out.paths, out.lengths, want)


@pytest.mark.parametrize("coop", [1, 33, 1 << 30], ids=["coop-all", "coop-33", "coop-off"])
def test_warp_cooperative_paths_bit_exact(small, coop):
    """MetaPath label scans and Node2Vec neighbour checks handed to the whole
    warp (every row at coop 1) give the same paths as the oracle."""
    g, G = small
    src = np.concatenate([synth.vertex_sources(g.nv), synth.sources(999, g.nv, seed=8)])
    old = G.tuning()
    try:
        G.set_tuning(coop_degree=coop, search_degree=max(coop, 33))
        for algo in (trw.METAPATH, trw.NODE2VEC):
            for kw in ([ALGO_KW[algo], {"n2v_p": 2.0, "n2v_q": 0.5}] if algo == trw.NODE2VEC else [ALGO_KW[algo]]):
                want = oracle_walk(g, algo, src, 60, seed=13, **kw)
                out = G.walk(algo, torch.from_numpy(src).cuda(), 60, seed=13, kernel=trw.KERNEL_PERSISTENT, **kw)
                torch.cuda.synchronize()
                assert_paths_equal(out.paths.cpu().numpy(), out.lengths.cpu().numpy(), want)
        reqs = [dict(algo=trw.METAPATH, sources=src, max_len=50, seed=3, schema=np.array([2, 4, 1], np.uint8)),
                dict(algo=trw.NODE2VEC, sources=src[:700], max_len=50, seed=4, n2v_p=0.5, n2v_q=2.0),
                dict(algo=trw.PPR, sources=src[:300], max_len=100, seed=5, ppr_stop=0.2)]
        outs = G.walk_batch(reqs)
        torch.cuda.synchronize()
        for r, o in zip(reqs, outs):
            kw = {k: r[k] for k in ("schema", "n2v_p", "n2v_q", "ppr_stop") if k in r}
            want = oracle_walk(g, r["algo"], r["sources"], r["max_len"], r["seed"], **kw)
            assert_paths_equal(o.paths.cpu().numpy(), o.lengths.cpu().numpy(), want)
    finally:
        G.set_tuning(**old)


@pytest.mark.parametrize("algo", [trw.DEEPWALK_WEIGHTED, trw.NODE2VEC, trw.PPR], ids=["weighted", "node2vec", "ppr"])
def test_pinned_host_outputs(small, algo):
    """Page-locked host outputs and sources (the end-to-end path) equal the oracle."""
    g, G = small
    src = np.concatenate([synth.vertex_sources(g.nv), synth.sources(321, g.nv, seed=12)])
    L = 80
    kw = ALGO_KW[algo]
    want = oracle_walk(g, algo, src, L, seed=17, alias=oracle_alias(SCALE) if algo == trw.DEEPWALK_WEIGHTED else None,
                       **kw)
    h_src = torch.from_numpy(src).pin_memory()
    h_paths = torch.full((src.shape[0], L + 1), -1, dtype=torch.int32).pin_memory()
    h_len = torch.full((src.shape[0],), -1, dtype=torch.int32).pin_memory()
    G.walk(algo, h_src.numpy(), L, seed=17, out_paths=h_paths.numpy(), out_lengths=h_len.numpy(), **kw)
    assert_paths_equal(h_paths.numpy(), h_len.numpy(), want)
    # endpoints into pinned memory too
    want = oracle_walk(g, algo, src, L, seed=18, alias=oracle_alias(SCALE) if algo == trw.DEEPWALK_WEIGHTED else None,
                       endpoints_only=True, **kw)
    h_end = torch.full((src.shape[0],), -1, dtype=torch.int32).pin_memory()
    G.walk(algo, h_src.numpy(), L, seed=18, endpoints=True, out_paths=h_end.numpy(), out_lengths=h_len.numpy(), **kw)
    assert_paths_equal(h_end.numpy(), h_len.numpy(), want, endpoints=True)


def test_auto_kernel_choice(small):
    """KERNEL_AUTO runs the one-launch kernel for a batch that fits in one
    resident wave, the persistent kernel beyond it; results are the oracle's
    either way."""
    g, G = small
    few = synth.sources(100, g.nv, seed=41)
    out = G.walk(trw.DEEPWALK, few, 30, seed=3)
    assert G.last_stats()["kernel"] == trw.KERNEL_PLAIN
    assert_paths_equal(out.paths, out.lengths, oracle_walk(g, trw.DEEPWALK, few, 30, seed=3))
    many = synth.sources(2_000_000, g.nv, seed=42)
    out = G.walk(trw.PPR, torch.from_numpy(many).cuda(), 50, seed=4, ppr_stop=0.2, endpoints=True)
    torch.cuda.synchronize()
    assert G.last_stats()["kernel"] == trw.KERNEL_PERSISTENT
    want = oracle_walk(g, trw.PPR, many, 50, seed=4, ppr_stop=0.2, endpoints_only=True)
    assert_paths_equal(out.paths.cpu().numpy(), out.lengths.cpu().numpy(), want, endpoints=True)
