"""Randomised parity (GPU only): many small seeded cases -- random graphs
(directed or not, with isolated vertices and zero weights), every algorithm
and sampler, random parameters, lengths, walks per source, walk offsets,
output modes and kernels -- each compared with the oracle walk for walk."""
import numpy as np
import pytest

import oracle
import paper_2107_11983_gb300 as trw
import synth
from gpu_common import assert_paths_equal

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N_CASES = 60


def random_graph(rng):
    nv = int(rng.integers(2, 400))
    m = int(rng.integers(1, 6 * nv))
    hub = rng.random() < 0.5
    u = rng.integers(0, nv, size=m)
    v = rng.integers(0, nv, size=m)
    if hub:  # a hub adjacent to a quarter of the vertices
        k = max(1, nv // 4)
        u = np.concatenate([u, np.zeros(k, np.int64)])
        v = np.concatenate([v, rng.integers(0, nv, size=k)])
    g = synth.from_edges(nv, list(zip(u.tolist(), v.tolist())), symmetric=bool(rng.random() < 0.6))
    w = rng.uniform(0.5, 50.0, size=g.ne).astype(np.float32)
    w[rng.random(g.ne) < 0.05] = 0.0  # some zero weights
    g.weights = w
    g.labels = rng.integers(0, 4, size=g.ne).astype(np.uint8)
    return g


def case_params(rng, g):
    choice = rng.integers(0, 10)
    kw = {}
    if choice in (0, 1):
        algo = trw.DEEPWALK
    elif choice == 2:
        algo = trw.PPR
        kw = {"ppr_stop": float(rng.choice([0.0, 0.05, 0.2, 0.5, 1.0]))}
    elif choice == 3:
        algo = trw.DEEPWALK_WEIGHTED
    elif choice in (4, 5):
        algo = trw.NODE2VEC
        kw = {"n2v_p": float(rng.choice([0.25, 0.5, 1.0, 2.0, 3.0])), "n2v_q": float(rng.choice([0.25, 0.5, 1.0, 2.0]))}
    elif choice == 6:
        algo = trw.METAPATH
        kw = {"schema": rng.integers(0, 4, size=int(rng.integers(1, 6))).astype(np.uint8)}
    elif choice == 7:
        algo = trw.NODE2VEC_WEIGHTED
        kw = {"n2v_p": 0.5, "n2v_q": 2.0, "max_weight": float(rng.choice([0.0, 60.0]))}
    else:
        algo = trw.DEEPWALK_WEIGHTED
        s = int(rng.choice([trw.SAMPLER_ITS, trw.SAMPLER_REJ]))
        kw = {"sampler": s}
    return algo, kw


@pytest.mark.parametrize("case", range(N_CASES))
def test_random_case(case):
    rng = np.random.default_rng(1000 + case)
    g = random_graph(rng)
    algo, kw = case_params(rng, g)
    G = trw.Graph(g.row_ptr, g.col, g.weights, g.labels)
    prep = trw.PREP_ALIAS | trw.PREP_ITS | trw.PREP_REJ
    if rng.random() < 0.5:
        prep |= trw.PREP_ROW_RECORDS | trw.PREP_NEIGHBOR_HASH | trw.PREP_LABEL_INDEX | trw.PREP_ITS_GUIDE
    G.prepare(prep)
    n = int(rng.integers(1, 300))
    src = rng.integers(0, g.nv, size=n).astype(np.int32)
    L = int(rng.choice([0, 1, 3, 17, 64]))
    wps = int(rng.integers(1, 4))
    off = int(rng.choice([0, 77, 2 ** 32 - n * wps]))
    seed = int(rng.integers(0, 2 ** 63))
    endpoints = bool(rng.random() < 0.2)
    kernel = int(rng.choice([trw.KERNEL_AUTO, trw.KERNEL_PLAIN, trw.KERNEL_PERSISTENT, trw.KERNEL_BSP]))
    okw = {k: v for k, v in kw.items() if k != "max_weight" or algo in (trw.DEEPWALK_WEIGHTED, trw.NODE2VEC_WEIGHTED)}
    oalgo = {trw.DEEPWALK: oracle.DEEPWALK, trw.DEEPWALK_WEIGHTED: oracle.DEEPWALK_WEIGHTED, trw.PPR: oracle.PPR,
             trw.NODE2VEC: oracle.NODE2VEC, trw.METAPATH: oracle.METAPATH,
             trw.NODE2VEC_WEIGHTED: oracle.NODE2VEC_WEIGHTED}[algo]
    tables = {}
    if algo in (trw.DEEPWALK_WEIGHTED, trw.NODE2VEC_WEIGHTED):
        tables = {"weights": g.weights, "its": oracle.prepare_its(g.row_ptr, g.weights),
                  "pmax": oracle.prepare_rej(g.row_ptr, g.weights)}
        if "sampler" not in kw:
            tables["alias"] = oracle.prepare_alias(g.row_ptr, g.weights)
    want = oracle.walk(g.row_ptr, g.col, oalgo, src, L, seed, labels=g.labels, walks_per_source=wps,
                       walk_offset=off, endpoints_only=endpoints, **okw, **tables)
    try:
        out = G.walk(algo, torch.from_numpy(src).cuda(), L, seed=seed, walks_per_source=wps, walk_offset=off,
                     endpoints=endpoints, kernel=kernel, **kw)
        torch.cuda.synchronize()
    except trw.TRWError as e:
        assert want.status != 0 and e.status == want.status, (e.status, want.status)
        return
    assert want.status == 0, want.status
    assert_paths_equal(out.paths.cpu().numpy(), out.lengths.cpu().numpy(), want, endpoints=endpoints)


def oracle_of_request(g, r, tables_all):
    algo, kw = r["algo"], dict(r["kw"])
    oalgo = {trw.DEEPWALK: oracle.DEEPWALK, trw.DEEPWALK_WEIGHTED: oracle.DEEPWALK_WEIGHTED, trw.PPR: oracle.PPR,
             trw.NODE2VEC: oracle.NODE2VEC, trw.METAPATH: oracle.METAPATH,
             trw.NODE2VEC_WEIGHTED: oracle.NODE2VEC_WEIGHTED}[algo]
    tables = {}
    if algo in (trw.DEEPWALK_WEIGHTED, trw.NODE2VEC_WEIGHTED):
        tables = dict(tables_all)
        if "sampler" in kw or algo == trw.NODE2VEC_WEIGHTED:
            tables.pop("alias")
    return oracle.walk(g.row_ptr, g.col, oalgo, r["src"], r["L"], r["seed"], labels=g.labels,
                       walks_per_source=r["wps"], endpoints_only=r["endpoints"], **kw, **tables)


@pytest.mark.parametrize("case", range(20))
def test_random_mixed_batch(case):
    rng = np.random.default_rng(5000 + case)
    g = random_graph(rng)
    G = trw.Graph(g.row_ptr, g.col, g.weights, g.labels)
    G.prepare(trw.PREP_ALIAS | trw.PREP_ITS | trw.PREP_REJ |
              (trw.PREP_ROW_RECORDS | trw.PREP_NEIGHBOR_HASH if rng.random() < 0.5 else 0))
    tables_all = {"weights": g.weights, "its": oracle.prepare_its(g.row_ptr, g.weights),
                  "pmax": oracle.prepare_rej(g.row_ptr, g.weights), "alias": oracle.prepare_alias(g.row_ptr, g.weights)}
    reqs = []
    for i in range(int(rng.integers(1, 7))):
        algo, kw = case_params(rng, g)
        if algo == trw.NODE2VEC_WEIGHTED and kw.get("max_weight") == 60.0:
            kw["max_weight"] = 0.0  # the REJ bounds: zero-weight rows are dead ends, never the trial cap
        reqs.append({"algo": algo, "kw": kw, "src": rng.integers(0, g.nv, size=int(rng.integers(1, 200))).astype(np.int32),
                     "L": int(rng.choice([0, 2, 9, 40])), "wps": int(rng.integers(1, 3)), "seed": int(rng.integers(0, 2 ** 40)),
                     "endpoints": bool(rng.random() < 0.3)})
    wants = [oracle_of_request(g, r, tables_all) for r in reqs]
    if any(w.status != 0 for w in wants):
        pytest.skip("a request of this draw fails in the oracle")
    outs = G.walk_batch([dict(algo=r["algo"], sources=r["src"], max_len=r["L"], seed=r["seed"],
                              walks_per_source=r["wps"], endpoints=r["endpoints"], **r["kw"]) for r in reqs])
    torch.cuda.synchronize()
    for r, o, w in zip(reqs, outs, wants):
        assert_paths_equal(o.paths.cpu().numpy(), o.lengths.cpu().numpy(), w, endpoints=r["endpoints"])
