"""The step-synchronous baseline (TRW_KERNEL_BSP, GPU only): one launch per
step over the live walkers gives the oracle's walks bit for bit, for every
algorithm and sampler, and reports its launch count."""
import numpy as np
import pytest

import oracle
import paper_2107_11983_gb300 as trw
import synth
from gpu_common import assert_paths_equal, oracle_alias, oracle_walk, rmat_graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SCHEMA = np.array([1, 3, 0, 4, 2], np.uint8)
CASES = {
    "deepwalk": (trw.DEEPWALK, 60, {}),
    "weighted": (trw.DEEPWALK_WEIGHTED, 60, {}),
    "ppr": (trw.PPR, 400, {"ppr_stop": 0.2}),
    "node2vec": (trw.NODE2VEC, 50, {"n2v_p": 0.5, "n2v_q": 2.0}),
    "metapath": (trw.METAPATH, 50, {"schema": SCHEMA}),
    "its": (trw.DEEPWALK_WEIGHTED, 40, {"sampler": trw.SAMPLER_ITS}),
    "rej": (trw.DEEPWALK_WEIGHTED, 40, {"sampler": trw.SAMPLER_REJ}),
    "orej": (trw.DEEPWALK_WEIGHTED, 40, {"sampler": trw.SAMPLER_OREJ, "max_weight": 100.0}),
}


@pytest.fixture(scope="module")
def graph():
    g = rmat_graph(12)
    G = trw.Graph(g.row_ptr, g.col, g.weights, g.labels)
    G.prepare(trw.PREP_ALIAS | trw.PREP_ITS | trw.PREP_REJ)
    return g, G


def want_of(g, algo, src, L, seed, kw, **extra):
    if "sampler" in kw:
        okw = dict(kw, weights=g.weights, its=oracle.prepare_its(g.row_ptr, g.weights),
                   pmax=oracle.prepare_rej(g.row_ptr, g.weights))
        return oracle_walk(g, algo, src, L, seed, **okw, **extra)
    return oracle_walk(g, algo, src, L, seed, alias=oracle_alias(12) if algo == trw.DEEPWALK_WEIGHTED else None,
                       **kw, **extra)


@pytest.mark.parametrize("case", list(CASES))
def test_bsp_matches_oracle(graph, case):
    g, G = graph
    algo, L, kw = CASES[case]
    src = np.concatenate([synth.vertex_sources(g.nv), synth.sources(999, g.nv, seed=4)])
    want = want_of(g, algo, src, L, 7, kw)
    out = G.walk(algo, torch.from_numpy(src).cuda(), L, seed=7, kernel=trw.KERNEL_BSP, **kw)
    torch.cuda.synchronize()
    assert_paths_equal(out.paths.cpu().numpy(), out.lengths.cpu().numpy(), want)
    st = G.last_stats()
    assert st["kernel"] == trw.KERNEL_BSP and st["moves"] == want.stats["moves"]
    # one launch per step while any walk is alive, plus the launch that creates the walkers;
    # a walk that stops early (coin, dead end, missing label) ends one launch after its last move
    longest = int(want.lengths.max()) - 1
    assert longest + 1 <= st["launches"] <= min(longest + 2, L + 1)


def test_bsp_host_buffers_endpoints_offsets(graph):
    g, G = graph
    src = synth.sources(1500, g.nv, seed=8)
    for algo, L, kw in (CASES["ppr"], CASES["node2vec"]):
        want = want_of(g, algo, src, L, 3, kw, walks_per_source=3, walk_offset=12345)
        out = G.walk(algo, src, L, seed=3, walks_per_source=3, walk_offset=12345, kernel=trw.KERNEL_BSP, **kw)
        assert_paths_equal(out.paths, out.lengths, want)
        ends = want_of(g, algo, src, L, 3, kw, endpoints_only=True)
        out = G.walk(algo, src, L, seed=3, endpoints=True, kernel=trw.KERNEL_BSP, **kw)
        assert_paths_equal(out.paths, out.lengths, ends, endpoints=True)


def test_bsp_edges_and_errors(graph):
    g, G = graph
    src = synth.sources(100, g.nv, seed=1)
    out = G.walk(trw.DEEPWALK, src, 0, seed=1, kernel=trw.KERNEL_BSP)
    assert np.array_equal(out.lengths, np.ones(100, np.int32)) and np.array_equal(out.paths[:, 0], src)
    assert G.last_stats()["launches"] == 1
    out = G.walk(trw.DEEPWALK, np.zeros(0, np.int32), 10, seed=1, kernel=trw.KERNEL_BSP)
    assert out.lengths.shape == (0,)
    bad = torch.from_numpy(np.array([0, 5, g.nv + 3], np.int32)).cuda()
    paths = torch.full((3, 11), -7, dtype=torch.int32, device="cuda")
    lens = torch.full((3,), -7, dtype=torch.int32, device="cuda")
    with pytest.raises(trw.TRWError) as e:
        G.walk(trw.DEEPWALK, bad, 10, seed=1, kernel=trw.KERNEL_BSP, out_paths=paths, out_lengths=lens)
    assert e.value.status == -1
    assert int((paths != -7).sum()) == 0 and int((lens != -7).sum()) == 0, "an invalid call wrote output"
    src_d = torch.from_numpy(src).cuda()
    with pytest.raises(trw.TRWError) as e:
        G.walk(trw.DEEPWALK, src_d, 10, seed=1, kernel=trw.KERNEL_BSP, sync=False)
    assert e.value.status == -1
