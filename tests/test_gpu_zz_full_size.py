"""Parity at the benchmark's full sizes (GPU only), in the launch
configuration bench.py times: the same synthetic graphs, tables, autotuning
and kernel choice, every walk of the batch on the GPU, compared vertex for
vertex with the oracle: every walk of DeepWalk on R-MAT s14 and of weighted
DeepWalk (ALIAS) on s22 (the oracle on all host cores, in contiguous walk
ranges); a sample of walks recomputed one by one (walk_offset = the walk's
index) for Node2Vec on s24 with the neighbour hash and row records, the mixed
batch (1M PPR endpoints + one MetaPath walk per vertex) on s23 with the label
index, and the largest graph, R-MAT s26 directed (1.07B edges): its weighted
DeepWalk batch and a served mix of the serving trace's requests."""
import argparse
import concurrent.futures as cf
import importlib.util
import os

import numpy as np
import pytest

import oracle
import paper_2107_11983_gb300 as trw
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N_SAMPLE = 300


def bench_module():
    spec = importlib.util.spec_from_file_location("bench_for_parity", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def check_sample(g, oalgo, src, L, seed, out, pick, endpoints=False, **kw):
    """out: the GPU's output of the whole batch; pick: walk indices to recompute."""
    idx = torch.from_numpy(np.asarray(pick, np.int64)).to(out.lengths.device)
    paths = out.paths[idx].cpu().numpy()
    lengths = out.lengths[idx].cpu().numpy()
    for r, i in enumerate(pick):
        i = int(i)
        w = oracle.walk(g.row_ptr, g.col, oalgo, src[i:i + 1], L, seed, labels=g.labels, walk_offset=i,
                        endpoints_only=endpoints, **kw)
        assert w.status == 0
        assert lengths[r] == w.lengths[0], (i, lengths[r], w.lengths[0])
        if endpoints:
            assert paths[r] == w.paths[0], i
        else:
            assert np.array_equal(paths[r, :lengths[r]], w.paths[0, :lengths[r]]), i


def oracle_alias_rows(g):
    """The oracle's ALIAS tables of every row, built in row ranges on every host
    core and concatenated: each row's table depends on that row alone, and its
    slot indices are local to the row."""
    cores = max(1, len(os.sched_getaffinity(0)))
    cuts = np.searchsorted(g.row_ptr, np.linspace(0, g.ne, cores + 1)).astype(np.int64)
    cuts[0], cuts[-1] = 0, g.nv
    cuts = np.maximum.accumulate(cuts)

    def part(j):
        lo, hi = int(cuts[j]), int(cuts[j + 1])
        e0, e1 = int(g.row_ptr[lo]), int(g.row_ptr[hi])
        return oracle.prepare_alias(g.row_ptr[lo:hi + 1] - e0, g.weights[e0:e1])

    with cf.ThreadPoolExecutor(cores) as ex:
        parts = list(ex.map(part, range(cores)))
    return oracle.AliasTables(np.concatenate([t.H for t in parts]), np.concatenate([t.A_first for t in parts]),
                              np.concatenate([t.A_second for t in parts]), np.concatenate([t.dead for t in parts]))


def check_all(g, oalgo, src, L, seed, out, **kw):
    """Every walk of the batch against the oracle, in contiguous walk ranges on
    every host core (the C walker runs outside the interpreter lock)."""
    n = src.shape[0]
    paths = out.paths.cpu().numpy()
    lengths = out.lengths.cpu().numpy()
    cores = max(1, len(os.sched_getaffinity(0)))
    bounds = np.linspace(0, n, cores + 1).astype(np.int64)

    def one(j):
        lo, hi = int(bounds[j]), int(bounds[j + 1])
        if lo == hi:
            return 0
        w = oracle.walk(g.row_ptr, g.col, oalgo, src[lo:hi], L, seed, labels=g.labels, walk_offset=lo, **kw)
        assert w.status == 0
        bad = np.nonzero(lengths[lo:hi] != w.lengths)[0]
        assert bad.size == 0, f"{bad.size} lengths differ, first walk {lo + bad[0]}"
        mask = np.arange(L + 1)[None, :] < w.lengths[:, None]
        rows = np.nonzero(((paths[lo:hi] != w.paths) & mask).any(axis=1))[0]
        assert rows.size == 0, f"{rows.size} paths differ, first walk {lo + rows[0]}"
        return int(w.stats["moves"])

    with cf.ThreadPoolExecutor(cores) as ex:
        moves = sum(ex.map(one, range(cores)))
    assert moves == int((out.lengths.to(torch.int64) - 1).sum().item())


@pytest.mark.parametrize("config", ["c1", "c2", "c3"])
def test_walk_configs_full_size(config):
    b = bench_module()
    wl = dict(b.WORKLOADS[config])
    args = argparse.Namespace(paper_paths=False)
    g = b.build_graph(wl)
    G = trw.Graph(g.row_ptr, g.col, g.weights, g.labels)
    algo = trw.ALGOS[wl["algo"]]
    alias = None
    if algo == trw.DEEPWALK_WEIGHTED:
        G.prepare(trw.PREP_ALIAS)
        alias = oracle.prepare_alias(g.row_ptr, g.weights)
    tables = b.tables_of(wl, args)
    if tables:
        G.prepare(tables)
    kw = b.walk_kwargs(wl)
    L = wl["max_len"]
    G.autotune(algo, L, **kw)
    src = synth.vertex_sources(g.nv)
    out = G.walk(algo, torch.from_numpy(src).cuda(), L, wl["seed"], **kw)  # the bench's kernel choice (AUTO)
    torch.cuda.synchronize()
    assert int((out.lengths.to(torch.int64) - 1).sum().item()) == G.last_stats()["moves"]
    oalgo = {trw.DEEPWALK: oracle.DEEPWALK, trw.DEEPWALK_WEIGHTED: oracle.DEEPWALK_WEIGHTED,
             trw.NODE2VEC: oracle.NODE2VEC}[algo]
    if config in ("c1", "c2"):
        check_all(g, oalgo, src, L, wl["seed"], out, alias=alias, **kw)
    else:
        pick = np.random.default_rng(11).choice(g.nv, 3 * N_SAMPLE, replace=False)
        check_sample(g, oalgo, src, L, wl["seed"], out, pick, alias=alias, **kw)


def test_largest_graph_full_size():
    """R-MAT s26 directed (the serving graph, 1.07B edges; dead ends): the
    weighted DeepWalk batch of one walk per vertex, and a served mix of the
    serving trace's first requests, each sampled against the oracle."""
    b = bench_module()
    wl = dict(b.WORKLOADS["c5"])
    args = argparse.Namespace(paper_paths=False)
    g = b.build_graph(wl)
    G = trw.Graph(g.row_ptr, g.col, g.weights, None)
    G.prepare(trw.PREP_ALIAS)
    G.prepare(b.tables_of(wl, args))
    G.autotune(trw.DEEPWALK_WEIGHTED, 80)
    alias = oracle_alias_rows(g)
    src = synth.vertex_sources(g.nv)
    out = G.walk(trw.DEEPWALK_WEIGHTED, torch.from_numpy(src).cuda(), 80, 1)
    torch.cuda.synchronize()
    assert int((out.lengths.to(torch.int64) - 1).sum().item()) == G.last_stats()["moves"]
    rng = np.random.default_rng(13)
    check_sample(g, oracle.DEEPWALK_WEIGHTED, src, 80, 1, out, rng.choice(g.nv, N_SAMPLE, replace=False), alias=alias)
    del out
    torch.cuda.empty_cache()
    # the serving trace's first 300 requests, queued at once (admission queues
    # them as memory allows); ten walks of each recomputed by the oracle
    _, reqs = b.serve_trace(g, 300, 2000.0)
    S = trw.Server(G, max_requests=1024)
    try:
        live, i = {}, 0
        while i < len(reqs) or live:
            while i < len(reqs):
                r = reqs[i]
                op, ol = b._out_buffers(torch, r, torch.device("cuda"))
                try:
                    rid = S.submit(r["algo"], torch.from_numpy(r["sources"]).cuda(), r["max_len"], r["seed"], op, ol,
                                   **b._req_kwargs(r))
                except trw.TRWError as e:
                    if e.status == -7:
                        break
                    raise
                live[rid] = (r, op, ol)
                i += 1
            for rid, st in S.reap():
                assert st == 0, (rid, st)
                r, op, ol = live.pop(rid)
                wps = r.get("walks_per_source", 1)
                nw = int(r["sources"].shape[0]) * wps
                oalgo = {trw.PPR: oracle.PPR, trw.DEEPWALK_WEIGHTED: oracle.DEEPWALK_WEIGHTED,
                         trw.NODE2VEC: oracle.NODE2VEC}[r["algo"]]
                kw = {k: r[k] for k in ("ppr_stop", "n2v_p", "n2v_q") if k in r}
                if r["algo"] == trw.DEEPWALK_WEIGHTED:
                    kw["alias"] = alias
                pick = rng.choice(nw, min(10, nw), replace=False)
                per_walk_src = r["sources"] if wps == 1 else np.repeat(r["sources"], wps)
                check_sample(g, oalgo, per_walk_src, r["max_len"], r["seed"], trw.WalkOutput(op, ol), pick,
                             endpoints=r.get("endpoints", False), **kw)
    finally:
        S.close()


def test_mixed_config_full_size():
    b = bench_module()
    wl = dict(b.WORKLOADS["c4"])
    g = b.build_graph(wl)
    G = trw.Graph(g.row_ptr, g.col, None, g.labels)
    G.prepare(trw.PREP_LABEL_INDEX)
    schema = synth.schema(5, 5, seed=1)
    G.autotune(trw.METAPATH, 80, schema=schema)
    ppr_src = synth.sources(1_000_000, g.nv, seed=1)
    mp_src = synth.vertex_sources(g.nv)
    reqs = [dict(algo=trw.PPR, sources=torch.from_numpy(ppr_src).cuda(), max_len=1000, seed=1, ppr_stop=0.2,
                 endpoints=True),
            dict(algo=trw.METAPATH, sources=torch.from_numpy(mp_src).cuda(), max_len=80, seed=1, schema=schema)]
    outs = G.walk_batch(reqs)
    torch.cuda.synchronize()
    rng = np.random.default_rng(12)
    check_sample(g, oracle.PPR, ppr_src, 1000, 1, outs[0], rng.choice(ppr_src.shape[0], N_SAMPLE, replace=False),
                 endpoints=True, ppr_stop=0.2)
    check_sample(g, oracle.METAPATH, mp_src, 80, 1, outs[1], rng.choice(g.nv, N_SAMPLE, replace=False),
                 schema=schema)
