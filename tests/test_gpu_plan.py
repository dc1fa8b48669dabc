"""Batch plans (trw_plan_*, GPU only): a mixed batch captured as a CUDA graph
and replayed gives the oracle's walks at every replay, follows seed changes,
and refuses an invalid source at launch without writing."""
import numpy as np
import pytest

import paper_2107_11983_gb300 as trw
import synth
from gpu_common import assert_paths_equal, oracle_alias, oracle_walk, rmat_graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SCALE = 12


def requests(g):
    return [
        dict(algo=trw.PPR, sources=synth.sources(3000, g.nv, seed=4), max_len=1000, seed=21, ppr_stop=0.2,
             endpoints=True),
        dict(algo=trw.METAPATH, sources=synth.vertex_sources(g.nv), max_len=80, seed=22,
             schema=np.array([0, 1, 2, 3, 4], np.uint8)),
        dict(algo=trw.DEEPWALK_WEIGHTED, sources=synth.sources(777, g.nv, seed=5), max_len=40, seed=23),
        dict(algo=trw.NODE2VEC, sources=synth.sources(555, g.nv, seed=6), max_len=30, seed=24, n2v_p=0.5, n2v_q=2.0),
        dict(algo=trw.DEEPWALK, sources=synth.sources(1, g.nv, seed=7), max_len=80, seed=25, walks_per_source=100),
    ]


def check(g, r, out, seed=None):
    kw = {k: r[k] for k in ("ppr_stop", "schema", "n2v_p", "n2v_q", "walks_per_source") if k in r}
    want = oracle_walk(g, r["algo"], r["sources"], r["max_len"], r["seed"] if seed is None else seed,
                       alias=oracle_alias(SCALE) if r["algo"] == trw.DEEPWALK_WEIGHTED else None,
                       endpoints_only=r.get("endpoints", False), **kw)
    assert_paths_equal(out.paths.cpu().numpy(), out.lengths.cpu().numpy(), want, endpoints=r.get("endpoints", False))
    return int((want.lengths.astype(np.int64) - 1).sum())


@pytest.mark.parametrize("prepared", [trw.PREP_ALIAS, trw.PREP_ALIAS | trw.PREP_LABEL_INDEX | trw.PREP_NEIGHBOR_HASH],
                         ids=["alias", "all-tables"])
def test_plan_replays_match_oracle(prepared):
    g = rmat_graph(SCALE)
    G = trw.Graph(g.row_ptr, g.col, g.weights, g.labels)
    G.prepare(prepared)
    reqs = requests(g)
    P = G.plan(reqs)
    try:
        P.launch()
        moves = P.sync()
        total = sum(check(g, r, o) for r, o in zip(reqs, P.outputs))
        assert moves == total
        first = [(o.paths.clone(), o.lengths.clone()) for o in P.outputs]
        for o in P.outputs:  # replays rewrite every output
            o.paths.fill_(-1)
            o.lengths.fill_(-1)
        torch.cuda.synchronize()
        for _ in range(4):
            P.launch()
        assert P.sync() == total
        for (p0, l0), o in zip(first, P.outputs):
            assert torch.equal(l0, o.lengths)
            if p0.dim() == 1:
                assert torch.equal(p0, o.paths)
            else:
                mask = torch.arange(p0.shape[1], device="cuda")[None, :] < l0[:, None]
                assert torch.equal(p0[mask], o.paths[mask])
        # new seeds take effect at the next launch
        P.set_seed(1, 777)
        P.set_seed(3, 2 ** 63 + 5)
        P.launch()
        P.sync()
        check(g, reqs[1], P.outputs[1], seed=777)
        check(g, reqs[3], P.outputs[3], seed=2 ** 63 + 5)
        check(g, reqs[0], P.outputs[0])
    finally:
        P.close()


def test_plan_on_a_stream_and_invalid_source():
    g = rmat_graph(SCALE)
    G = trw.Graph(g.row_ptr, g.col, None, None)
    bad = synth.sources(1000, g.nv, seed=3)
    bad[517] = g.nv  # out of range
    reqs = [dict(algo=trw.DEEPWALK, sources=synth.sources(2000, g.nv, seed=2), max_len=20, seed=1),
            dict(algo=trw.DEEPWALK, sources=bad, max_len=20, seed=2)]
    P = G.plan(reqs)
    try:
        for o in P.outputs:
            o.paths.fill_(-1)
            o.lengths.fill_(-1)
        s = torch.cuda.Stream()
        torch.cuda.synchronize()
        P.launch(stream=s)
        with pytest.raises(trw.TRWError) as e:
            P.sync()
        assert e.value.status == -1
        for o in P.outputs:  # nothing written
            assert bool((o.lengths == -1).all()) and bool((o.paths == -1).all())
    finally:
        P.close()
    # a valid plan on a side stream
    ok = [dict(algo=trw.PPR, sources=synth.sources(5000, g.nv, seed=9), max_len=100, seed=3, ppr_stop=0.2)]
    P = G.plan(ok)
    try:
        s = torch.cuda.Stream()
        P.launch(stream=s)
        P.sync()
        check(g, ok[0], P.outputs[0])
    finally:
        P.close()


@pytest.mark.parametrize("algo", [trw.DEEPWALK_WEIGHTED, trw.NODE2VEC, trw.METAPATH], ids=["weighted", "node2vec", "metapath"])
def test_single_request_plan(algo):
    """A one-request plan runs the algorithm's own kernel; a seed change
    re-captures it."""
    g = rmat_graph(SCALE)
    G = trw.Graph(g.row_ptr, g.col, g.weights, g.labels)
    G.prepare()
    kw = {trw.NODE2VEC: dict(n2v_p=0.5, n2v_q=2.0), trw.METAPATH: dict(schema=np.array([2, 0, 4], np.uint8))}.get(algo, {})
    r = dict(algo=algo, sources=synth.sources(5000, g.nv, seed=12), max_len=50, seed=31, **kw)
    P = G.plan([r])
    try:
        P.launch()
        moves = P.sync()
        assert moves == check(g, r, P.outputs[0])
        P.set_seed(0, 4242)
        P.launch()
        P.launch()
        P.sync()
        check(g, r, P.outputs[0], seed=4242)
    finally:
        P.close()
