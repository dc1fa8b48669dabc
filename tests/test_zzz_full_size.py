"""Parity at the benchmark's full sizes (GPU only), in the launch
configuration bench.py times: the same synthetic graphs, tables, autotuning
and kernel choice, every walk of the batch on the GPU, and a sample of walks
recomputed one by one by the oracle (walk_offset = the walk's index) and
compared vertex for vertex: DeepWalk on R-MAT s14, weighted DeepWalk (ALIAS)
on s22, Node2Vec on s24 with the neighbour hash and row records, and the
mixed batch (1M PPR endpoints + one MetaPath walk per vertex) on s23 with the
label index."""
import argparse
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
    pick = np.random.default_rng(11).choice(g.nv, N_SAMPLE, replace=False)
    oalgo = {trw.DEEPWALK: oracle.DEEPWALK, trw.DEEPWALK_WEIGHTED: oracle.DEEPWALK_WEIGHTED,
             trw.NODE2VEC: oracle.NODE2VEC}[algo]
    check_sample(g, oalgo, src, L, wl["seed"], out, pick, alias=alias, **kw)


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
