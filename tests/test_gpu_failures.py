"""Failure paths made on the host (GPU only): a call on the wrong device, an
allocation that fails, a bounded wait that runs out.  None of them faults or
hangs the GPU: the wrong device is a pretended one (the library's test hook
changes only what its device check compares), the failed allocation is
injected in the library's allocation gate before cudaMalloc is called, and the
drain's wait is the host's.  After each failure the graph or server must still
give the oracle's walks."""
import ctypes

import numpy as np
import pytest

import paper_2107_11983_gb300 as trw
import synth
from gpu_common import assert_paths_equal, oracle_alias, oracle_walk, rmat_graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SCALE = 12
ERR_INVALID, ERR_OOM, ERR_NOT_PREPARED, ERR_TIMEOUT = -1, -2, -3, -5


@pytest.fixture(autouse=True)
def hooks_off():
    yield
    trw.fail_allocs(-1)
    trw.pretend_device(-1)


def _raises(status, fn, *a, **kw):
    with pytest.raises(trw.TRWError) as ei:
        fn(*a, **kw)
    assert ei.value.status == status, str(ei.value)
    return str(ei.value)


def _deepwalk_matches(g, G, n=500, seed=3):
    src = synth.sources(n, g.nv, seed=seed)
    got = G.walk(trw.DEEPWALK, src, 40, seed)
    assert_paths_equal(got.paths, got.lengths, oracle_walk(g, trw.DEEPWALK, src, 40, seed))


def _weighted_matches(g, G, n=500, seed=4):
    src = synth.sources(n, g.nv, seed=seed)
    got = G.walk(trw.DEEPWALK_WEIGHTED, src, 40, seed)
    assert_paths_equal(got.paths, got.lengths, oracle_walk(g, trw.DEEPWALK_WEIGHTED, src, 40, seed,
                                                           alias=oracle_alias(SCALE)))


def test_wrong_device_refused_before_any_launch():
    g = rmat_graph(SCALE)
    G = trw.Graph(g.row_ptr, g.col, g.weights, g.labels)
    G.prepare()
    S = trw.Server(G)
    dev = torch.cuda.current_device()
    src = torch.from_numpy(synth.sources(256, g.nv, seed=5)).cuda()
    op = torch.full((256, 41), -7, dtype=torch.int32, device="cuda")
    ol = torch.full((256,), -7, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    try:
        trw.pretend_device(dev + 1)
        msg = _raises(ERR_INVALID, G.walk, trw.DEEPWALK, src, 40, 1, out_paths=op, out_lengths=ol)
        assert "current device" in msg
        _raises(ERR_INVALID, G.prepare, trw.PREP_ROW_RECORDS)
        _raises(ERR_INVALID, G.walk_batch, [dict(algo=trw.DEEPWALK, sources=src, max_len=40, seed=1)])
        _raises(ERR_INVALID, G.autotune, trw.DEEPWALK, 40)
        _raises(ERR_INVALID, trw.Plan, G, [dict(algo=trw.DEEPWALK, sources=src, max_len=40, seed=1)])
        _raises(ERR_INVALID, trw.Server, G)
        _raises(ERR_INVALID, S.submit, trw.DEEPWALK, src, 40, 1, op, ol)
        _raises(ERR_INVALID, S.drain, 1000)
        lib = trw.load_library()
        n = 1
        arr = (ctypes.c_void_p * n)()
        st = lib.trw_walk_batch_noalloc(G.handle, n, (ctypes.c_int * n)(), None, arr, (ctypes.c_int64 * n)(),
                                        (ctypes.c_int32 * n)(), (ctypes.c_uint64 * n)(), arr, arr, None)
        assert st == ERR_INVALID and b"current device" in lib.trw_last_error()
        torch.cuda.synchronize()
        assert bool((op == -7).all()) and bool((ol == -7).all()), "a refused call wrote output"
    finally:
        trw.pretend_device(-1)
    _deepwalk_matches(g, G)
    _weighted_matches(g, G)
    S.drain(10000)
    S.close()


def test_prepare_out_of_memory_leaves_graph_usable():
    g = rmat_graph(SCALE)
    G = trw.Graph(g.row_ptr, g.col, g.weights, g.labels)
    # fail the alias tables themselves (after=0), then the first scratch array
    # (after=1: the tables exist from then on), then the last one (after=2)
    for after in range(3):
        trw.fail_allocs(after)
        _raises(ERR_OOM, G.prepare, trw.PREP_ALIAS)
        trw.fail_allocs(-1)
        _raises(ERR_NOT_PREPARED, G.walk, trw.DEEPWALK_WEIGHTED, synth.sources(8, g.nv, seed=1), 10, 1)
        _deepwalk_matches(g, G, seed=10 + after)
    # the optional tables: a failed build adds nothing, the walks stay the oracle's
    for flag in (trw.PREP_LABEL_INDEX, trw.PREP_NEIGHBOR_HASH, trw.PREP_ROW_RECORDS, trw.PREP_ITS, trw.PREP_REJ,
                 trw.PREP_ITS_GUIDE):
        before = G.device_bytes()
        trw.fail_allocs(0)
        _raises(ERR_OOM, G.prepare, flag)
        trw.fail_allocs(-1)
        assert G.device_bytes() == before
        _deepwalk_matches(g, G, seed=flag)
    G.prepare()
    _weighted_matches(g, G)


def test_graph_load_out_of_memory():
    g = rmat_graph(SCALE)
    for after in (0, 1, 3):
        trw.fail_allocs(after)
        _raises(ERR_OOM, trw.Graph, g.row_ptr, g.col, g.weights, g.labels)
    trw.fail_allocs(-1)
    G = trw.Graph(g.row_ptr, g.col, g.weights, g.labels)
    _deepwalk_matches(g, G)


def test_serve_out_of_memory_leaves_server_usable():
    g = rmat_graph(SCALE)
    G = trw.Graph(g.row_ptr, g.col, g.weights, g.labels)
    G.prepare()
    for after in (0, 2, 5):
        trw.fail_allocs(after)
        _raises(ERR_OOM, trw.Server, G)
    trw.fail_allocs(-1)
    S = trw.Server(G)
    try:
        src_h = synth.sources(3000, g.nv, seed=7)
        src = torch.from_numpy(src_h).cuda()
        op = torch.full((3000, 41), -1, dtype=torch.int32, device="cuda")
        ol = torch.full((3000,), -1, dtype=torch.int32, device="cuda")
        # device sources: admission copies them to pinned memory for the range
        # check; that buffer's allocation fails and nothing is queued
        trw.fail_allocs(0)
        _raises(ERR_OOM, S.submit, trw.DEEPWALK_WEIGHTED, src, 40, 9, op, ol)
        trw.fail_allocs(-1)
        rid = S.submit(trw.DEEPWALK_WEIGHTED, src, 40, 9, op, ol)
        S.drain(60000)
        assert S.poll(rid) == trw.OK
        assert_paths_equal(op.cpu().numpy(), ol.cpu().numpy(),
                           oracle_walk(g, trw.DEEPWALK_WEIGHTED, src_h, 40, 9, alias=oracle_alias(SCALE)))
    finally:
        S.close()


def test_drain_timeout_then_completion():
    g = rmat_graph(SCALE)
    G = trw.Graph(g.row_ptr, g.col, g.weights, g.labels)
    S = trw.Server(G)
    try:
        n = 1 << 20  # about 8e7 moves: milliseconds of walking
        src_h = synth.sources(n, g.nv, seed=8)
        src = torch.from_numpy(src_h).cuda()
        op = torch.full((n, 81), -1, dtype=torch.int32, device="cuda")
        ol = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        rid = S.submit(trw.DEEPWALK, src, 80, 12, op, ol)
        msg = _raises(ERR_TIMEOUT, S.drain, 0)
        assert "still running" in msg
        S.drain(60000)
        assert S.poll(rid) == trw.OK
        # walk i of the request is keyed on index i: the first 2000 walks, and
        # 50 more anywhere in the request recomputed with their own index
        got_p, got_l = op.cpu().numpy(), ol.cpu().numpy()
        want = oracle_walk(g, trw.DEEPWALK, src_h[:2000], 80, 12)
        assert_paths_equal(got_p[:2000], got_l[:2000], want)
        for i in np.random.default_rng(1).choice(n, 50, replace=False):
            w1 = oracle_walk(g, trw.DEEPWALK, src_h[i:i + 1], 80, 12, walk_offset=int(i))
            assert_paths_equal(got_p[i:i + 1], got_l[i:i + 1], w1)
    finally:
        S.close()
