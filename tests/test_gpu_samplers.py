"""Weighted DeepWalk under ITS, REJ and O-REJ (Section 2.3), GPU only: the
prepared tables equal the oracle's, and every walk equals the oracle's bit
for bit in every kernel, with and without row records, in mixed batches,
plans and the server; zero-weight rows, clamped bounds, extreme weights and
the error paths behave as documented."""
import functools
import time

import numpy as np
import pytest

import oracle
import paper_2107_11983_gb300 as trw
import synth
from gpu_common import assert_paths_equal, rmat_graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SAMPLERS = {"its": trw.SAMPLER_ITS, "rej": trw.SAMPLER_REJ, "orej": trw.SAMPLER_OREJ}
BOUND = 100.0  # synth weights lie in [1, 100)


@functools.lru_cache(maxsize=None)
def oracle_tables(scale: int, symmetric: bool = True):
    g = rmat_graph(scale, symmetric=symmetric)
    return oracle.prepare_its(g.row_ptr, g.weights), oracle.prepare_rej(g.row_ptr, g.weights)


def oracle_sampled(g, sampler, sources, max_len, seed, tables, max_weight=BOUND, **kw):
    cdf, pm = tables
    res = oracle.walk(g.row_ptr, g.col, oracle.DEEPWALK_WEIGHTED, sources, max_len, seed, sampler=sampler,
                      weights=g.weights, its=cdf, pmax=pm, max_weight=max_weight, **kw)
    return res


def test_tables_match_oracle():
    for scale, sym in ((11, True), (12, False)):
        g = rmat_graph(scale, symmetric=sym)
        G = trw.Graph(g.row_ptr, g.col, g.weights)
        G.prepare(trw.PREP_ITS | trw.PREP_REJ)
        cdf, pm = G.debug_sampler_tables()
        want_cdf, want_pm = oracle_tables(scale, sym)
        assert np.array_equal(cdf, want_cdf)
        assert np.array_equal(pm, want_pm)
    G2 = trw.Graph(g.row_ptr, g.col, g.weights)
    with pytest.raises(trw.TRWError) as e:
        G2.debug_sampler_tables()
    assert e.value.status == -3


def its_records_want(g, cdf):
    """Guided ITS records recomputed on the host from the oracle's prefix sums:
    U_j = floor((P'_j 2^64 - 1) / S) (0 where P'_j = 0); the first candidate of
    cell k is the smallest j with max(ceil(k 2^64 / d), 1) <= U_j, the last
    one the first of cell k + 1 (d - 1 for the last cell); -1 in a row whose
    weights are all zero."""
    M = 1 << 64
    rows = []
    for v in range(g.nv):
        lo, hi = int(g.row_ptr[v]), int(g.row_ptr[v + 1])
        d = hi - lo
        if d == 0:
            continue
        P = [int(x) for x in cdf[lo:hi]]
        S = P[-1]
        U = [0 if p == 0 or S == 0 else ((p << 64) - 1) // S for p in P]
        Ua = np.array(U, dtype=np.uint64)
        if S == 0:
            first = [-1] * d
            last = [-1] * d
        else:
            cells = [max(-(-k * M // d), 1) for k in range(d)]
            first = [int(np.searchsorted(Ua, np.uint64(c), side="left")) for c in cells]
            last = first[1:] + [d - 1]
        for j in range(d):
            c = int(g.col[lo + j])
            rows.append([U[j] & 0xFFFFFFFF, U[j] >> 32, c, int(g.row_ptr[c]), int(g.row_ptr[c + 1] - g.row_ptr[c]),
                         first[j] & 0xFFFFFFFF, last[j] & 0xFFFFFFFF, 0])
    return np.array(rows, dtype=np.uint64).astype(np.uint32)


def test_its_guide_records_match_host():
    for scale, sym in ((10, True), (11, False)):
        g = rmat_graph(scale, symmetric=sym)
        G = trw.Graph(g.row_ptr, g.col, g.weights)
        G.prepare(trw.PREP_ITS_GUIDE)
        got = G.debug_its_records()
        want = its_records_want(g, oracle.prepare_its(g.row_ptr, g.weights))
        assert np.array_equal(got, want)
    with pytest.raises(trw.TRWError) as e:
        trw.Graph(g.row_ptr, g.col, g.weights).debug_its_records()
    assert e.value.status == -3


@pytest.mark.parametrize("records", [False, True], ids=["plain-tables", "records"])
@pytest.mark.parametrize("kernel", [trw.KERNEL_PLAIN, trw.KERNEL_PERSISTENT], ids=["plain", "persistent"])
@pytest.mark.parametrize("name", list(SAMPLERS))
def test_sampler_walks_match_oracle(name, kernel, records):
    g = rmat_graph(12)
    src = np.concatenate([synth.vertex_sources(g.nv), synth.sources(1237, g.nv, seed=3)])
    want = oracle_sampled(g, SAMPLERS[name], src, 60, 17, oracle_tables(12))
    assert want.status == 0
    preps = [trw.PREP_ITS | trw.PREP_REJ] + ([trw.PREP_ITS_GUIDE] if name == "its" else [])
    for prep in preps:  # ITS: the prefix-sum search, then the guided records alone
        G = trw.Graph(g.row_ptr, g.col, g.weights)
        G.prepare(prep | (trw.PREP_ROW_RECORDS if records else 0))
        out = G.walk(trw.DEEPWALK_WEIGHTED, torch.from_numpy(src).cuda(), 60, seed=17, kernel=kernel,
                     sampler=SAMPLERS[name], max_weight=BOUND)
        torch.cuda.synchronize()
        assert_paths_equal(out.paths.cpu().numpy(), out.lengths.cpu().numpy(), want)
        assert G.last_stats()["moves"] == want.stats["moves"]


@pytest.mark.parametrize("name", list(SAMPLERS))
def test_sampler_endpoints_offsets_and_host_buffers(name):
    g = rmat_graph(11, symmetric=False)
    G = trw.Graph(g.row_ptr, g.col, g.weights)
    G.prepare(trw.PREP_REJ | (trw.PREP_ITS_GUIDE if name == "its" else 0))
    src = synth.sources(700, g.nv, seed=9)
    off = 2 ** 32 - 700 * 3
    want = oracle_sampled(g, SAMPLERS[name], src, 40, 2 ** 64 - 5, oracle_tables(11, False), walks_per_source=3,
                          walk_offset=off)
    out = G.walk(trw.DEEPWALK_WEIGHTED, src, 40, seed=2 ** 64 - 5, walks_per_source=3, walk_offset=off,
                 sampler=SAMPLERS[name], max_weight=BOUND)
    assert_paths_equal(out.paths, out.lengths, want)
    ends = oracle_sampled(g, SAMPLERS[name], src, 40, 3, oracle_tables(11, False), endpoints_only=True)
    out = G.walk(trw.DEEPWALK_WEIGHTED, src, 40, seed=3, endpoints=True, sampler=SAMPLERS[name], max_weight=BOUND)
    assert_paths_equal(out.paths, out.lengths, ends, endpoints=True)


def test_orej_bound_below_the_largest_weight():
    # P = 40 < max w: darts on heavier edges always hit (their threshold clamps to 2^32)
    g = rmat_graph(11)
    G = trw.Graph(g.row_ptr, g.col, g.weights)
    src = synth.vertex_sources(g.nv)
    for bound in (40.0, 1.0, 1e9):
        want = oracle_sampled(g, trw.SAMPLER_OREJ, src, 30, 4, (None, None), max_weight=bound)
        assert want.status == 0
        out = G.walk(trw.DEEPWALK_WEIGHTED, src, 30, seed=4, sampler=trw.SAMPLER_OREJ, max_weight=bound)
        assert_paths_equal(out.paths, out.lengths, want)


def test_zero_weight_rows_and_extreme_weights():
    # hub 0 with zero, tiny, huge and clamped weights; vertex 5's edges are all zero
    edges = [(0, k) for k in range(1, 9)] + [(k, 0) for k in range(1, 9)] + [(5, 6), (5, 7), (2, 3), (3, 2)]
    g = synth.from_edges(9, edges, symmetric=False)
    wmap = {(0, k): w for k, w in zip(range(1, 9), [0.0, 1e-5, 3.0, 70000.0, 2.5 / 65536, 1e30, 65535.998, 0.0])}
    wmap.update({(k, 0): 1.0 for k in range(1, 9)})
    wmap.update({(5, 0): 0.0, (5, 6): 0.0, (5, 7): 0.0, (2, 3): 1.0, (3, 2): 4.0})
    g.weights = np.array([wmap[(v, int(c))] for v in range(9) for c in g.col[g.row_ptr[v]:g.row_ptr[v + 1]]],
                         np.float32)
    tables = (oracle.prepare_its(g.row_ptr, g.weights), oracle.prepare_rej(g.row_ptr, g.weights))
    G = trw.Graph(g.row_ptr, g.col, g.weights)
    G.prepare(trw.PREP_ITS | trw.PREP_REJ | trw.PREP_ROW_RECORDS)
    cdf, pm = G.debug_sampler_tables()
    assert np.array_equal(cdf, tables[0]) and np.array_equal(pm, tables[1])
    Gg = trw.Graph(g.row_ptr, g.col, g.weights)
    Gg.prepare(trw.PREP_ITS_GUIDE)
    assert np.array_equal(Gg.debug_its_records(), its_records_want(g, tables[0]))
    src = np.array([0, 1, 2, 3, 4, 6, 7, 8, 0, 0], np.int32)
    for name, graph in (("its", G), ("its", Gg), ("rej", G)):
        want = oracle_sampled(g, SAMPLERS[name], src, 25, 6, tables, walks_per_source=300)
        assert want.status == 0
        for kernel in (trw.KERNEL_PLAIN, trw.KERNEL_PERSISTENT):
            out = graph.walk(trw.DEEPWALK_WEIGHTED, src, 25, seed=6, walks_per_source=300, kernel=kernel,
                             sampler=SAMPLERS[name])
            assert_paths_equal(out.paths, out.lengths, want)
    dead = oracle_sampled(g, trw.SAMPLER_ITS, np.array([5], np.int32), 4, 1, tables)
    assert dead.lengths[0] == 1
    # O-REJ cannot see that row 5 has no positive weight: the trial cap ends the call
    with pytest.raises(trw.TRWError) as e:
        G.walk(trw.DEEPWALK_WEIGHTED, np.array([5], np.int32), 4, seed=1, sampler=trw.SAMPLER_OREJ, max_weight=2.0)
    assert e.value.status == -6
    assert oracle_sampled(g, trw.SAMPLER_OREJ, np.array([5], np.int32), 4, 1, tables, max_weight=2.0).status == -6


@pytest.mark.parametrize("guide", [False, True], ids=["its-search", "its-guided"])
def test_mixed_batch_plan_and_server(guide):
    g = rmat_graph(12)
    G = trw.Graph(g.row_ptr, g.col, g.weights, g.labels)
    G.prepare(trw.PREP_ALIAS | trw.PREP_REJ | (trw.PREP_ITS_GUIDE if guide else trw.PREP_ITS))
    tables = oracle_tables(12)
    reqs = []
    for i, (name, s) in enumerate(SAMPLERS.items()):
        reqs.append(dict(algo=trw.DEEPWALK_WEIGHTED, sources=synth.sources(2000 + 300 * i, g.nv, seed=20 + i),
                         max_len=50, seed=30 + i, sampler=s, max_weight=BOUND))
    reqs.append(dict(algo=trw.PPR, sources=synth.sources(3000, g.nv, seed=40), max_len=200, seed=41, ppr_stop=0.2,
                     endpoints=True))
    reqs.append(dict(algo=trw.NODE2VEC, sources=synth.sources(1500, g.nv, seed=42), max_len=40, seed=43, n2v_p=0.5,
                     n2v_q=2.0))

    def want_of(r):
        if r["algo"] == trw.DEEPWALK_WEIGHTED:
            return oracle_sampled(g, r["sampler"], r["sources"], r["max_len"], r["seed"], tables)
        kw = {k: v for k, v in r.items() if k in ("ppr_stop", "n2v_p", "n2v_q")}
        return oracle.walk(g.row_ptr, g.col, r["algo"], r["sources"], r["max_len"], r["seed"],
                           endpoints_only=r.get("endpoints", False), **kw)

    wants = [want_of(r) for r in reqs]
    outs = G.walk_batch(reqs)
    torch.cuda.synchronize()
    for r, o, w in zip(reqs, outs, wants):
        assert_paths_equal(o.paths.cpu().numpy(), o.lengths.cpu().numpy(), w, endpoints=r.get("endpoints", False))
    plan = G.plan(reqs)
    for _ in range(2):
        plan.launch()
        plan.sync()
        for r, o, w in zip(reqs, plan.outputs, wants):
            assert_paths_equal(o.paths.cpu().numpy(), o.lengths.cpu().numpy(), w, endpoints=r.get("endpoints", False))
    plan.close()
    S = trw.Server(G, max_requests=64)
    try:
        for r, w in zip(reqs[:3], wants[:3]):
            src = torch.from_numpy(r["sources"]).cuda()
            n = src.shape[0]
            op = torch.empty((n, r["max_len"] + 1), dtype=torch.int32, device="cuda")
            ol = torch.empty(n, dtype=torch.int32, device="cuda")
            rid = S.submit(r["algo"], src, r["max_len"], r["seed"], op, ol, sampler=r["sampler"],
                           max_weight=r["max_weight"])
            t0 = time.time()
            while S.poll(rid) == trw.PENDING:
                assert time.time() - t0 < 60, "request did not finish"
            assert_paths_equal(op.cpu().numpy(), ol.cpu().numpy(), w)
    finally:
        S.close()


def test_full_size_sampled_parity():
    # R-MAT s20 (about 1M vertices, 32M edges): one walk per vertex in the
    # launch configuration of the benchmark; 2000 sampled walks against the oracle
    g = rmat_graph(20)
    G = trw.Graph(g.row_ptr, g.col, g.weights)
    G.prepare(trw.PREP_ITS | trw.PREP_REJ | trw.PREP_ROW_RECORDS)
    src = torch.arange(g.nv, dtype=torch.int32, device="cuda")
    pick = np.sort(np.random.default_rng(5).choice(g.nv, 2000, replace=False)).astype(np.int64)
    cdf, pm = oracle_tables(20)
    runs = list(SAMPLERS.items()) + [("its-guided", trw.SAMPLER_ITS)]
    for name, s in runs:
        if name == "its-guided":
            G.prepare(trw.PREP_ITS_GUIDE)
        out = G.walk(trw.DEEPWALK_WEIGHTED, src, 80, seed=99, sampler=s, max_weight=BOUND,
                     kernel=trw.KERNEL_PERSISTENT)
        torch.cuda.synchronize()
        paths = out.paths.cpu().numpy()[pick]
        lens = out.lengths.cpu().numpy()[pick]
        for i, v in enumerate(pick if name.startswith("its") else pick[:200]):
            w = oracle.walk(g.row_ptr, g.col, oracle.DEEPWALK_WEIGHTED, [int(v)], 80, 99, sampler=s,
                            weights=g.weights, its=cdf, pmax=pm, max_weight=BOUND, walk_offset=int(v))
            assert w.status == 0
            assert lens[i] == w.lengths[0], (name, int(v))
            assert np.array_equal(paths[i, :lens[i]], w.paths[0, :lens[i]]), (name, int(v))


def test_errors():
    g = rmat_graph(10)
    G = trw.Graph(g.row_ptr, g.col, g.weights)
    src = synth.sources(10, g.nv, seed=1)
    for s, prep in ((trw.SAMPLER_ITS, "ITS"), (trw.SAMPLER_REJ, "REJ")):
        with pytest.raises(trw.TRWError) as e:
            G.walk(trw.DEEPWALK_WEIGHTED, src, 5, seed=1, sampler=s)
        assert e.value.status == -3 and prep in str(e.value)
    for bad in (0.0, -1.0, float("nan"), float("inf"), 1e-6):
        with pytest.raises(trw.TRWError) as e:
            G.walk(trw.DEEPWALK_WEIGHTED, src, 5, seed=1, sampler=trw.SAMPLER_OREJ, max_weight=bad)
        assert e.value.status == -1
    with pytest.raises(trw.TRWError) as e:
        G.walk(trw.DEEPWALK, src, 5, seed=1, sampler=trw.SAMPLER_ITS)
    assert e.value.status == -1
    with pytest.raises(trw.TRWError) as e:
        G.walk(trw.DEEPWALK_WEIGHTED, src, 5, seed=1, sampler=7)
    assert e.value.status == -1
    U = trw.Graph(g.row_ptr, g.col)
    with pytest.raises(trw.TRWError) as e:
        U.prepare(trw.PREP_ITS)
    assert e.value.status == -1
    with pytest.raises(trw.TRWError) as e:
        U.walk(trw.DEEPWALK_WEIGHTED, src, 5, seed=1, sampler=trw.SAMPLER_OREJ, max_weight=2.0)
    assert e.value.status == -1
