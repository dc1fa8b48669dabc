"""Neighbour hash (TRW_PREP_NEIGHBOR_HASH, GPU only).

IsNeighbor as the kernels evaluate it is checked against set membership
computed here from the CSR arrays, with and without the hash, and Node2Vec
walks that use it against the oracle, whose IsNeighbor is the binary search
of Section 4.  Walks must be bit-identical with and without the hash."""
import time

import numpy as np
import pytest

import paper_2107_11983_gb300 as trw
import synth
from gpu_common import assert_paths_equal, oracle_alias, oracle_walk, rmat_graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N2V = dict(n2v_p=0.5, n2v_q=2.0)


def membership_cases(g, rng, n_random=200_000):
    """Every edge of the longest rows, random edges, random pairs (mostly
    non-edges) and near misses (a neighbour id plus or minus one)."""
    deg = np.diff(g.row_ptr)
    u_parts, v_parts = [], []
    for u in np.argsort(deg)[::-1][:20]:
        lo, hi = g.row_ptr[u], g.row_ptr[u + 1]
        u_parts.append(np.full(hi - lo, u, np.int32))
        v_parts.append(g.col[lo:hi])
    e = rng.integers(0, g.ne, n_random)
    src_of = np.repeat(np.arange(g.nv, dtype=np.int32), deg)
    u_parts += [src_of[e], rng.integers(0, g.nv, n_random).astype(np.int32), src_of[e]]
    v_parts += [g.col[e], rng.integers(0, g.nv, n_random).astype(np.int32),
                np.clip(g.col[e] + rng.choice([-1, 1], n_random), 0, g.nv - 1).astype(np.int32)]
    u = np.concatenate(u_parts).astype(np.int32)
    v = np.concatenate(v_parts).astype(np.int32)
    edges = set(zip(src_of.tolist(), g.col.tolist()))
    want = np.array([(a, b) in edges for a, b in zip(u.tolist(), v.tolist())])
    return u, v, want


@pytest.mark.parametrize("symmetric", [True, False], ids=["sym", "directed"])
def test_is_neighbor_matches_sets(symmetric):
    g = rmat_graph(12, symmetric=symmetric)
    u, v, want = membership_cases(g, np.random.default_rng(3))
    assert want.any() and not want.all()
    G = trw.Graph(g.row_ptr, g.col, None, None)
    assert np.array_equal(G.debug_is_neighbor(u, v), want)  # binary search
    before = G.device_bytes()
    G.prepare(trw.PREP_NEIGHBOR_HASH)
    assert G.device_bytes() > before
    assert np.array_equal(G.debug_is_neighbor(u, v), want)  # hash for rows of 8 or more
    G.prepare(trw.PREP_NEIGHBOR_HASH)  # already built: nothing changes
    assert np.array_equal(G.debug_is_neighbor(u, v), want)


@pytest.mark.parametrize("kernel", [trw.KERNEL_PLAIN, trw.KERNEL_PERSISTENT], ids=["plain", "persistent"])
def test_hashed_node2vec_matches_oracle(kernel):
    g = rmat_graph(12)
    G = trw.Graph(g.row_ptr, g.col, None, None)
    G.prepare(trw.PREP_NEIGHBOR_HASH)
    src = np.concatenate([synth.vertex_sources(g.nv), synth.sources(1237, g.nv, seed=3)])
    for p, q, seed in [(0.5, 2.0, 7), (2.0, 0.5, 8), (1.0, 1.0, 9), (0.25, 4.0, 10)]:
        want = oracle_walk(g, trw.NODE2VEC, src, 80, seed=seed, n2v_p=p, n2v_q=q)
        out = G.walk(trw.NODE2VEC, torch.from_numpy(src).cuda(), 80, seed=seed, kernel=kernel, n2v_p=p, n2v_q=q)
        torch.cuda.synchronize()
        assert_paths_equal(out.paths.cpu().numpy(), out.lengths.cpu().numpy(), want)


def test_hashed_and_searched_walks_identical():
    g = rmat_graph(14)
    src = synth.sources(50_000, g.nv, seed=8)
    plain = trw.Graph(g.row_ptr, g.col, None, None)
    hashed = trw.Graph(g.row_ptr, g.col, None, None)
    hashed.prepare(trw.PREP_NEIGHBOR_HASH)
    a = plain.walk(trw.NODE2VEC, src, 60, seed=5, walks_per_source=2, **N2V)
    b = hashed.walk(trw.NODE2VEC, src, 60, seed=5, walks_per_source=2, **N2V)
    assert np.array_equal(a.lengths, b.lengths)
    mask = np.arange(61)[None, :] < a.lengths[:, None]
    assert np.array_equal(a.paths[mask], b.paths[mask])


def test_hashed_mixed_batch_and_serve():
    g = rmat_graph(12)
    G = trw.Graph(g.row_ptr, g.col, g.weights, g.labels)
    G.prepare(trw.PREP_ALIAS | trw.PREP_LABEL_INDEX | trw.PREP_NEIGHBOR_HASH)
    reqs = [
        dict(algo=trw.NODE2VEC, sources=synth.sources(4000, g.nv, seed=6), max_len=50, seed=24, **N2V),
        dict(algo=trw.METAPATH, sources=synth.sources(999, g.nv, seed=9), max_len=33, seed=25,
             schema=np.array([4, 4, 2], np.uint8)),
        dict(algo=trw.DEEPWALK_WEIGHTED, sources=synth.sources(777, g.nv, seed=5), max_len=40, seed=23),
        dict(algo=trw.NODE2VEC, sources=synth.sources(1, g.nv, seed=7), max_len=80, seed=26, walks_per_source=300,
             n2v_p=2.0, n2v_q=0.5),
    ]

    def check(r, paths, lengths):
        kw = {k: r[k] for k in ("n2v_p", "n2v_q", "schema", "walks_per_source") if k in r}
        want = oracle_walk(g, r["algo"], r["sources"], r["max_len"], r["seed"],
                           alias=oracle_alias(12) if r["algo"] == trw.DEEPWALK_WEIGHTED else None, **kw)
        assert_paths_equal(paths, lengths, want)

    outs = G.walk_batch(reqs)
    torch.cuda.synchronize()
    for r, o in zip(reqs, outs):
        check(r, o.paths.cpu().numpy(), o.lengths.cpu().numpy())

    S = trw.Server(G, max_requests=16)
    try:
        live = []
        for r in reqs:
            n = r["sources"].shape[0] * r.get("walks_per_source", 1)
            op = torch.full((n, r["max_len"] + 1), -1, dtype=torch.int32, device="cuda")
            ol = torch.full((n,), -1, dtype=torch.int32, device="cuda")
            kw = {k: r[k] for k in ("n2v_p", "n2v_q", "schema", "walks_per_source") if k in r}
            live.append((r, S.submit(r["algo"], r["sources"], r["max_len"], r["seed"], op, ol, **kw), op, ol))
        for r, rid, op, ol in live:
            t = time.time()
            while S.poll(rid) == trw.PENDING:
                assert time.time() - t < 60
                time.sleep(0.0005)
            check(r, op.cpu().numpy(), ol.cpu().numpy())
    finally:
        S.close()


def test_hash_on_tiny_and_empty_rows():
    # rows below the hash's minimum degree keep the binary search; a star row
    # and isolated vertices
    edges = [(0, k) for k in range(1, 40)] + [(1, 2), (2, 3), (3, 1), (5, 0)]
    g = synth.from_edges(45, edges, symmetric=True)
    G = trw.Graph(g.row_ptr, g.col, None, None)
    G.prepare(trw.PREP_NEIGHBOR_HASH)
    u = np.repeat(np.arange(45, dtype=np.int32), 45)
    v = np.tile(np.arange(45, dtype=np.int32), 45)
    es = set(zip(np.repeat(np.arange(45), np.diff(g.row_ptr)).tolist(), g.col.tolist()))
    want = np.array([(a, b) in es for a, b in zip(u.tolist(), v.tolist())])
    assert np.array_equal(G.debug_is_neighbor(u, v), want)
    src = np.arange(45, dtype=np.int32).repeat(20)
    out = G.walk(trw.NODE2VEC, src, 30, seed=2, **N2V)
    assert_paths_equal(out.paths, out.lengths, oracle_walk(g, trw.NODE2VEC, src, 30, seed=2, **N2V))
    with pytest.raises(trw.TRWError):
        G.debug_is_neighbor(np.array([45], np.int32), np.array([0], np.int32))
