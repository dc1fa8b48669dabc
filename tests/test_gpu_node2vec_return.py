"""Node2Vec's return-only darts (GPU only).  With row records on a graph
without weights, each record's aux word is the position of the edge's source
in its destination's row; a Node2Vec dart whose word lies at or past both
non-return thresholds can only be accepted as a return to the previous vertex,
so the kernels decide it from that position without reading the candidate.
The positions must be exact and the walks the oracle's, for parameters that do
and do not leave such darts, on symmetric and directed graphs (where the edge
back may be missing), in every kernel and with or without the neighbour hash;
on a weighted graph the aux word is the weight and the walks stay exact."""
import numpy as np
import pytest

import oracle
import paper_2107_11983_gb300 as trw
import synth
from gpu_common import assert_paths_equal, oracle_walk, rmat_graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def expected_weight_words(weights):
    """The records' aux word on a weighted graph: the oracle's integer weight,
    as the int32 with the same bits."""
    q = np.array([oracle.quantize_weight(float(w)) for w in weights], dtype=np.int64)
    return q.astype(np.uint32).view(np.int32)


def expected_records(g, weights=None):
    """dst, its row offset and degree, W_e, and the position of the source in
    the destination's row (-1: absent), by searchsorted on the host."""
    nv = g.nv
    src = np.repeat(np.arange(nv, dtype=np.int64), np.diff(g.row_ptr))
    dst = g.col.astype(np.int64)
    rev = np.full(g.ne, -1, dtype=np.int64)
    for e in range(g.ne):
        lo, hi = g.row_ptr[dst[e]], g.row_ptr[dst[e] + 1]
        k = lo + np.searchsorted(g.col[lo:hi], src[e])
        if k < hi and g.col[k] == src[e]:
            rev[e] = k - lo
    return dst, g.row_ptr[dst], g.row_ptr[dst + 1] - g.row_ptr[dst], rev


@pytest.mark.parametrize("symmetric", [True, False], ids=["sym", "directed"])
def test_row_record_reverse_positions(symmetric):
    g = rmat_graph(11, symmetric=symmetric)
    G = trw.Graph(g.row_ptr, g.col, None, None)
    G.prepare(trw.PREP_ROW_RECORDS)
    rec = G.debug_row_records()
    dst, off, deg, rev = expected_records(g)
    assert np.array_equal(rec[:, 0], dst)
    assert np.array_equal(rec[:, 1], off)
    assert np.array_equal(rec[:, 2], deg)
    assert np.array_equal(rec[:, 3], rev)
    if symmetric:
        assert (rev >= 0).all()
    else:
        assert (rev == -1).any() and (rev >= 0).any()


PARAMS = [(0.5, 2.0), (2.0, 0.5), (1.0, 1.0), (0.25, 4.0), (4.0, 0.25), (1.0, 0.5), (0.5, 1.0)]


@pytest.mark.parametrize("prep", [trw.PREP_ROW_RECORDS, trw.PREP_ROW_RECORDS | trw.PREP_NEIGHBOR_HASH],
                         ids=["records", "records+hash"])
@pytest.mark.parametrize("kernel", [trw.KERNEL_PLAIN, trw.KERNEL_PERSISTENT, trw.KERNEL_BSP],
                         ids=["plain", "persistent", "bsp"])
@pytest.mark.parametrize("symmetric", [True, False], ids=["sym", "directed"])
def test_node2vec_return_only_darts_match_oracle(symmetric, kernel, prep):
    g = rmat_graph(12, symmetric=symmetric)
    G = trw.Graph(g.row_ptr, g.col, None, None)
    G.prepare(prep)
    src = np.concatenate([synth.vertex_sources(g.nv), synth.sources(1500, g.nv, seed=4)])
    for i, (p, q) in enumerate(PARAMS):
        want = oracle_walk(g, trw.NODE2VEC, src, 50, seed=20 + i, n2v_p=p, n2v_q=q)
        out = G.walk(trw.NODE2VEC, torch.from_numpy(src).cuda(), 50, seed=20 + i, kernel=kernel, n2v_p=p, n2v_q=q)
        torch.cuda.synchronize()
        assert_paths_equal(out.paths.cpu().numpy(), out.lengths.cpu().numpy(), want)


def test_node2vec_return_only_darts_in_mixed_batch_and_weighted_graph():
    """Node2Vec beside other algorithms in one launch, on a weighted graph
    (the records' aux word is the weight: no return positions)."""
    g = rmat_graph(12)
    G = trw.Graph(g.row_ptr, g.col, g.weights, None)
    G.prepare(trw.PREP_ALIAS | trw.PREP_ROW_RECORDS)
    rec = G.debug_row_records()
    assert np.array_equal(rec[:, 3], expected_weight_words(g.weights))
    srcs = [synth.sources(3000, g.nv, seed=s) for s in (5, 6, 7)]
    reqs = [dict(algo=trw.NODE2VEC, sources=torch.from_numpy(srcs[0]).cuda(), max_len=40, seed=31, n2v_p=0.5,
                 n2v_q=2.0),
            dict(algo=trw.DEEPWALK, sources=torch.from_numpy(srcs[1]).cuda(), max_len=40, seed=32),
            dict(algo=trw.NODE2VEC, sources=torch.from_numpy(srcs[2]).cuda(), max_len=40, seed=33, n2v_p=4.0,
                 n2v_q=0.25)]
    outs = G.walk_batch(reqs)
    torch.cuda.synchronize()
    for r, s, o in zip(reqs, srcs, outs):
        kw = {k: r[k] for k in ("n2v_p", "n2v_q") if k in r}
        want = oracle_walk(g, r["algo"], s, 40, r["seed"], **kw)
        assert_paths_equal(o.paths.cpu().numpy(), o.lengths.cpu().numpy(), want)
