"""Compact path output (TRW_OUT_COMPACT, GPU only): the walks' vertices one
after the other, equal to the oracle's paths concatenated, for host and
device buffers, one slice and several; invalid uses are refused and write
nothing."""
import numpy as np
import pytest

import paper_2107_11983_gb300 as trw
import synth
from gpu_common import oracle_walk, rmat_graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def concat(want):
    mask = np.arange(want.paths.shape[1])[None, :] < want.lengths[:, None]
    return want.paths[mask]


@pytest.fixture(scope="module")
def graph():
    g = rmat_graph(12)
    G = trw.Graph(g.row_ptr, g.col, g.weights, g.labels)
    G.prepare(trw.PREP_ALIAS)
    return g, G


CASES = {
    "ppr": (trw.PPR, 60, {"ppr_stop": 0.2}),
    "deepwalk": (trw.DEEPWALK, 20, {}),
    "node2vec": (trw.NODE2VEC, 15, {"n2v_p": 0.5, "n2v_q": 2.0}),
}


@pytest.mark.parametrize("device", [False, True], ids=["host", "device"])
@pytest.mark.parametrize("case", list(CASES))
def test_compact_matches_oracle(graph, case, device):
    g, G = graph
    algo, L, kw = CASES[case]
    src = synth.sources(3000, g.nv, seed=2)
    want = oracle_walk(g, algo, src, L, 5, walks_per_source=2, **kw)
    s = torch.from_numpy(src).cuda() if device else src
    for kernel in (trw.KERNEL_PLAIN, trw.KERNEL_PERSISTENT):
        out = G.walk(algo, s, L, seed=5, walks_per_source=2, compact=True, kernel=kernel, **kw)
        paths = out.paths.cpu().numpy() if device else out.paths
        lens = out.lengths.cpu().numpy() if device else out.lengths
        assert np.array_equal(lens, want.lengths)
        assert np.array_equal(paths, concat(want))


def test_compact_many_slices(graph):
    # 2^19 + 300 walks: two slices and a ragged tail; isolated sources make short rows
    g, G = graph
    src = synth.sources((1 << 19) + 300, g.nv, seed=7)
    want = oracle_walk(g, trw.DEEPWALK, src, 6, 3)
    out = G.walk(trw.DEEPWALK, src, 6, seed=3, compact=True)
    assert np.array_equal(out.lengths, want.lengths)
    assert np.array_equal(out.paths, concat(want))
    assert G.last_stats()["launches"] == 2
    assert G.last_stats()["moves"] == int((want.lengths - 1).sum())
    # the caller's own pinned buffer, larger than needed: entries past the total stay as they were
    cap = src.shape[0] * 7
    host = torch.full((cap,), -5, dtype=torch.int32).pin_memory()
    lens = torch.empty(src.shape[0], dtype=torch.int32).pin_memory()
    G.walk(trw.DEEPWALK, src, 6, seed=3, compact=True, out_paths=host.numpy(), out_lengths=lens.numpy())
    total = int(want.lengths.sum())
    assert np.array_equal(host.numpy()[:total], concat(want)) and bool((host.numpy()[total:] == -5).all())


def test_compact_refusals(graph):
    g, G = graph
    src = synth.sources(100, g.nv, seed=1)
    d = torch.from_numpy(src).cuda()
    with pytest.raises(trw.TRWError) as e:
        G.walk(trw.DEEPWALK, d, 5, seed=1, compact=True, sync=False)
    assert e.value.status == -1
    with pytest.raises(trw.TRWError) as e:
        G.walk(trw.DEEPWALK, d, 5, seed=1, compact=True, kernel=trw.KERNEL_BSP)
    assert e.value.status == -1
    with pytest.raises(trw.TRWError) as e:
        _batch_with_compact(G, src)
    assert e.value.status == -1
    bad = torch.from_numpy(np.array([0, g.nv + 2], np.int32)).cuda()
    paths = torch.full((2 * 6,), -7, dtype=torch.int32, device="cuda")
    lens = torch.full((2,), -7, dtype=torch.int32, device="cuda")
    with pytest.raises(trw.TRWError) as e:
        G.walk(trw.DEEPWALK, bad, 5, seed=1, compact=True, out_paths=paths, out_lengths=lens)
    assert e.value.status == -1
    assert int((paths != -7).sum()) == 0 and int((lens != -7).sum()) == 0


def _batch_with_compact(G, src):
    """trw_walk_batch with a compact request, through the C ABI."""
    import ctypes
    lib = trw.load_library()
    p, _ = trw._params(trw.DEEPWALK, 0.2, 1.0, 1.0, None, 1, False, 0)
    p.out_mode = trw.OUT_COMPACT
    d = torch.from_numpy(src).cuda()
    op = torch.empty(src.shape[0] * 6, dtype=torch.int32, device="cuda")
    ol = torch.empty(src.shape[0], dtype=torch.int32, device="cuda")
    params = (trw._Params * 1)(p)
    st = lib.trw_walk_batch(G.handle, 1, (ctypes.c_int * 1)(trw.DEEPWALK), params,
                            (ctypes.c_void_p * 1)(d.data_ptr()), (ctypes.c_int64 * 1)(src.shape[0]),
                            (ctypes.c_int32 * 1)(5), (ctypes.c_uint64 * 1)(1), (ctypes.c_void_p * 1)(op.data_ptr()),
                            (ctypes.c_void_p * 1)(ol.data_ptr()), None, 1)
    if st != 0:
        raise trw.TRWError(st, "batch")
