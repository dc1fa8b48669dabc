"""Row records (TRW_PREP_ROW_RECORDS, GPU only): NAIVE moves and O-REJ
candidates read one record carrying the destination's row.  Walks must equal
the oracle's, and be identical with and without the records, alone and
combined with the other prepared tables, in every kernel."""
import time

import numpy as np
import pytest

import paper_2107_11983_gb300 as trw
import synth
from gpu_common import assert_paths_equal, oracle_alias, oracle_walk, rmat_graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = {
    "deepwalk": (trw.DEEPWALK, 80, {}),
    "ppr": (trw.PPR, 300, {"ppr_stop": 0.2}),
    "node2vec": (trw.NODE2VEC, 60, {"n2v_p": 0.5, "n2v_q": 2.0}),
    "node2vec-ab": (trw.NODE2VEC, 60, {"n2v_p": 2.0, "n2v_q": 0.5}),
}


@pytest.mark.parametrize("prep", [trw.PREP_ROW_RECORDS, trw.PREP_ROW_RECORDS | trw.PREP_NEIGHBOR_HASH],
                         ids=["records", "records+hash"])
@pytest.mark.parametrize("kernel", [trw.KERNEL_PLAIN, trw.KERNEL_PERSISTENT], ids=["plain", "persistent"])
@pytest.mark.parametrize("case", list(CASES))
def test_row_record_walks_match_oracle(case, kernel, prep):
    algo, L, kw = CASES[case]
    g = rmat_graph(12)
    G = trw.Graph(g.row_ptr, g.col, None, None)
    G.prepare(prep)
    src = np.concatenate([synth.vertex_sources(g.nv), synth.sources(1237, g.nv, seed=3)])
    want = oracle_walk(g, algo, src, L, seed=11, **kw)
    out = G.walk(algo, torch.from_numpy(src).cuda(), L, seed=11, kernel=kernel, **kw)
    torch.cuda.synchronize()
    assert_paths_equal(out.paths.cpu().numpy(), out.lengths.cpu().numpy(), want)


@pytest.mark.parametrize("symmetric", [True, False], ids=["sym", "directed"])
def test_row_records_identical_walks(symmetric):
    g = rmat_graph(14, symmetric=symmetric)
    src = synth.sources(40_000, g.nv, seed=8)
    plain = trw.Graph(g.row_ptr, g.col, None, None)
    rec = trw.Graph(g.row_ptr, g.col, None, None)
    rec.prepare(trw.PREP_ROW_RECORDS)
    assert rec.device_bytes() >= plain.device_bytes() + 16 * g.ne
    for algo, L, kw in CASES.values():
        a = plain.walk(algo, src, L, seed=5, walks_per_source=2, **kw)
        b = rec.walk(algo, src, L, seed=5, walks_per_source=2, **kw)
        assert np.array_equal(a.lengths, b.lengths)
        mask = np.arange(L + 1)[None, :] < a.lengths[:, None]
        assert np.array_equal(a.paths[mask], b.paths[mask])


def test_all_tables_mixed_batch_and_serve():
    g = rmat_graph(12)
    G = trw.Graph(g.row_ptr, g.col, g.weights, g.labels)
    G.prepare(trw.PREP_ALL)
    reqs = [
        dict(algo=trw.PPR, sources=synth.sources(3000, g.nv, seed=4), max_len=1000, seed=21, ppr_stop=0.2,
             endpoints=True),
        dict(algo=trw.DEEPWALK, sources=synth.sources(2000, g.nv, seed=1), max_len=80, seed=20),
        dict(algo=trw.METAPATH, sources=synth.sources(999, g.nv, seed=9), max_len=33, seed=25,
             schema=np.array([4, 4, 2], np.uint8)),
        dict(algo=trw.DEEPWALK_WEIGHTED, sources=synth.sources(777, g.nv, seed=5), max_len=40, seed=23),
        dict(algo=trw.NODE2VEC, sources=synth.sources(4000, g.nv, seed=6), max_len=50, seed=24, n2v_p=0.5,
             n2v_q=2.0),
    ]

    def check(r, paths, lengths):
        kw = {k: r[k] for k in ("ppr_stop", "n2v_p", "n2v_q", "schema", "walks_per_source") if k in r}
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
            n = r["sources"].shape[0]
            shape = (n,) if r.get("endpoints") else (n, r["max_len"] + 1)
            op = torch.full(shape, -1, dtype=torch.int32, device="cuda")
            ol = torch.full((n,), -1, dtype=torch.int32, device="cuda")
            kw = {k: r[k] for k in ("ppr_stop", "n2v_p", "n2v_q", "schema", "endpoints") if k in r}
            live.append((r, S.submit(r["algo"], r["sources"], r["max_len"], r["seed"], op, ol, **kw), op, ol))
        for r, rid, op, ol in live:
            t = time.time()
            while S.poll(rid) == trw.PENDING:
                assert time.time() - t < 60
                time.sleep(0.0005)
            check(r, op.cpu().numpy(), ol.cpu().numpy())
    finally:
        S.close()
