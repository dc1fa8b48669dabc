"""Weighted Node2Vec (Eq. 1 times the edge weight, GPU only): every walk
equals the oracle's, with the REJ bounds and with a caller's bound, in every
kernel, with and without the optional tables and the warp-cooperative
search, in mixed batches, plans and the server."""
import time

import numpy as np
import pytest

import oracle
import paper_2107_11983_gb300 as trw
import synth
from gpu_common import assert_paths_equal, rmat_graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

KW = {"n2v_p": 0.5, "n2v_q": 2.0}


def want_of(g, src, L, seed, max_weight=0.0, p=0.5, q=2.0, **extra):
    res = oracle.walk(g.row_ptr, g.col, oracle.NODE2VEC_WEIGHTED, src, L, seed, n2v_p=p, n2v_q=q,
                      weights=g.weights, pmax=oracle.prepare_rej(g.row_ptr, g.weights), max_weight=max_weight,
                      **extra)
    assert res.status == 0
    return res


@pytest.mark.parametrize("bound", [0.0, 100.0, 60.0], ids=["rej-bounds", "max-weight", "low-max-weight"])
@pytest.mark.parametrize("prep", [0, trw.PREP_ROW_RECORDS | trw.PREP_NEIGHBOR_HASH], ids=["paper", "tables"])
@pytest.mark.parametrize("symmetric", [True, False], ids=["sym", "directed"])
def test_weighted_node2vec_matches_oracle(bound, prep, symmetric):
    g = rmat_graph(12, symmetric=symmetric)
    G = trw.Graph(g.row_ptr, g.col, g.weights)
    G.prepare(trw.PREP_REJ | prep)
    src = np.concatenate([synth.vertex_sources(g.nv), synth.sources(777, g.nv, seed=2)])
    want = want_of(g, src, 40, 13, max_weight=bound)
    for kernel in (trw.KERNEL_PLAIN, trw.KERNEL_PERSISTENT, trw.KERNEL_BSP):
        out = G.walk(trw.NODE2VEC_WEIGHTED, torch.from_numpy(src).cuda(), 40, seed=13, kernel=kernel,
                     max_weight=bound, **KW)
        torch.cuda.synchronize()
        assert_paths_equal(out.paths.cpu().numpy(), out.lengths.cpu().numpy(), want)
        assert G.last_stats()["moves"] == want.stats["moves"]


def test_warp_search_and_hub():
    # a hub adjacent to most vertices: long rows of prev go to the warp search
    n = 20_001
    leaves = np.arange(1, n, dtype=np.int64)
    ring = np.stack([leaves, np.roll(leaves, -1)], axis=1)
    edges = np.concatenate([np.stack([np.zeros(n - 1, np.int64), leaves], axis=1), ring[::2]])
    g = synth.from_edges(n, edges.tolist(), symmetric=True)
    g.weights = synth.edge_weights(g)
    G = trw.Graph(g.row_ptr, g.col, g.weights)
    G.prepare(trw.PREP_REJ)
    G.set_tuning(search_degree=64)
    src = np.concatenate([np.zeros(200, np.int32), synth.sources(2000, n, seed=4)])
    for bound in (0.0, 100.0):
        want = want_of(g, src, 30, 3, max_weight=bound, p=2.0, q=0.5)
        out = G.walk(trw.NODE2VEC_WEIGHTED, src, 30, seed=3, kernel=trw.KERNEL_PERSISTENT, max_weight=bound,
                     n2v_p=2.0, n2v_q=0.5)
        assert_paths_equal(out.paths, out.lengths, want)


def test_equal_weights_reduce_to_node2vec():
    g = rmat_graph(11)
    w = np.full(g.ne, 2.5, np.float32)
    G = trw.Graph(g.row_ptr, g.col, w)
    G.prepare(trw.PREP_REJ)
    src = synth.vertex_sources(g.nv)
    base = G.walk(trw.NODE2VEC, src, 30, seed=5, **KW)
    for bound in (0.0, 2.5):
        out = G.walk(trw.NODE2VEC_WEIGHTED, src, 30, seed=5, max_weight=bound, **KW)
        assert np.array_equal(out.lengths, base.lengths)
        mask = np.arange(31)[None, :] < base.lengths[:, None]
        assert np.array_equal(out.paths[mask], base.paths[mask])


@pytest.mark.parametrize("bound", [0.0, 100.0], ids=["rej-bounds", "max-weight"])
def test_mixed_batch_plan_server(bound):
    g = rmat_graph(12)
    G = trw.Graph(g.row_ptr, g.col, g.weights, g.labels)
    G.prepare(trw.PREP_ALIAS | trw.PREP_REJ)
    reqs = [dict(algo=trw.NODE2VEC_WEIGHTED, sources=synth.sources(3000, g.nv, seed=9), max_len=40, seed=21,
                 max_weight=bound, walks_per_source=2, **KW),
            dict(algo=trw.NODE2VEC, sources=synth.sources(2000, g.nv, seed=10), max_len=40, seed=22, **KW),
            dict(algo=trw.PPR, sources=synth.sources(2000, g.nv, seed=11), max_len=300, seed=23, ppr_stop=0.2,
                 endpoints=True)]
    wants = [want_of(g, reqs[0]["sources"], 40, 21, max_weight=bound, walks_per_source=2),
             oracle.walk(g.row_ptr, g.col, oracle.NODE2VEC, reqs[1]["sources"], 40, 22, **KW),
             oracle.walk(g.row_ptr, g.col, oracle.PPR, reqs[2]["sources"], 300, 23, ppr_stop=0.2,
                         endpoints_only=True)]
    outs = G.walk_batch(reqs)
    torch.cuda.synchronize()
    for r, o, w in zip(reqs, outs, wants):
        assert_paths_equal(o.paths.cpu().numpy(), o.lengths.cpu().numpy(), w, endpoints=r.get("endpoints", False))
    plan = G.plan(reqs)
    plan.launch()
    plan.sync()
    for r, o, w in zip(reqs, plan.outputs, wants):
        assert_paths_equal(o.paths.cpu().numpy(), o.lengths.cpu().numpy(), w, endpoints=r.get("endpoints", False))
    plan.close()
    S = trw.Server(G, max_requests=16)
    try:
        src = torch.from_numpy(reqs[0]["sources"]).cuda()
        op = torch.empty((6000, 41), dtype=torch.int32, device="cuda")
        ol = torch.empty(6000, dtype=torch.int32, device="cuda")
        rid = S.submit(trw.NODE2VEC_WEIGHTED, src, 40, 21, op, ol, max_weight=bound, walks_per_source=2, **KW)
        t0 = time.time()
        while S.poll(rid) == trw.PENDING:
            assert time.time() - t0 < 60
        assert_paths_equal(op.cpu().numpy(), ol.cpu().numpy(), wants[0])
    finally:
        S.close()


def test_errors():
    g = rmat_graph(10)
    src = synth.sources(10, g.nv, seed=1)
    G = trw.Graph(g.row_ptr, g.col, g.weights)
    with pytest.raises(trw.TRWError) as e:
        G.walk(trw.NODE2VEC_WEIGHTED, src, 5, seed=1, **KW)  # no max_weight and no REJ bounds
    assert e.value.status == -3
    for bad in (-1.0, float("nan"), float("inf"), 1e-7):
        with pytest.raises(trw.TRWError) as e:
            G.walk(trw.NODE2VEC_WEIGHTED, src, 5, seed=1, max_weight=bad, **KW)
        assert e.value.status == -1
    U = trw.Graph(g.row_ptr, g.col)
    with pytest.raises(trw.TRWError) as e:
        U.walk(trw.NODE2VEC_WEIGHTED, src, 5, seed=1, max_weight=2.0, **KW)
    assert e.value.status == -1
    with pytest.raises(trw.TRWError) as e:
        G.walk(trw.NODE2VEC_WEIGHTED, src, 5, seed=1, max_weight=2.0, sampler=trw.SAMPLER_REJ, **KW)
    assert e.value.status == -1
