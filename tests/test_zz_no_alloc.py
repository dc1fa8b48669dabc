"""The no-allocation batch walk (GPU only).

trw_walk_batch_noalloc is for callers that must not allocate device memory
during a call: code that runs while the caller's own memory pool owns the
free device memory, code under an allocator that must see every allocation,
or a path where cudaMalloc/cudaFree would synchronise the device.  These tests
call it through the C ABI and check, on two calls in a row that share the
library's fixed scratch array, its paths and lengths against the oracle and
against trw_walk_batch, bit for bit (the tolerance of every walk test here);
that a call leaves the device's free memory unchanged and still succeeds when
every allocation the library makes is forced to fail; and the NULL stream.
Collected last, so that a run that stops at a failure here has already run
every other test."""
import ctypes
import gc

import numpy as np
import pytest

import oracle
import paper_2107_11983_gb300 as trw
import synth
from gpu_common import assert_paths_equal, oracle_alias, rmat_graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _requests(g):
    return [
        dict(algo=trw.PPR, sources=synth.sources(2000, g.nv, seed=4), max_len=1000, seed=21, ppr_stop=0.2,
             endpoints=True),
        dict(algo=trw.METAPATH, sources=synth.vertex_sources(g.nv), max_len=40, seed=22,
             schema=np.array([0, 1, 2, 3, 4], np.uint8)),
        dict(algo=trw.DEEPWALK_WEIGHTED, sources=synth.sources(777, g.nv, seed=5), max_len=40, seed=23),
        dict(algo=trw.NODE2VEC, sources=synth.sources(555, g.nv, seed=6), max_len=30, seed=24, n2v_p=0.5, n2v_q=2.0),
        dict(algo=trw.DEEPWALK, sources=synth.sources(3, g.nv, seed=7), max_len=80, seed=25, walks_per_source=100),
        dict(algo=trw.DEEPWALK_WEIGHTED, sources=synth.sources(900, g.nv, seed=8), max_len=30, seed=26,
             sampler=trw.SAMPLER_ITS),
        dict(algo=trw.DEEPWALK_WEIGHTED, sources=synth.sources(900, g.nv, seed=9), max_len=30, seed=27,
             sampler=trw.SAMPLER_OREJ, max_weight=100.0),
        dict(algo=trw.NODE2VEC_WEIGHTED, sources=synth.sources(600, g.nv, seed=10), max_len=30, seed=28, n2v_p=0.5,
             n2v_q=2.0, max_weight=100.0),
    ]


def _call_noalloc(G, reqs, stream="torch"):
    """Marshal the requests and call the C entry point directly (stream: the
    current torch stream, or None for the NULL stream)."""
    lib = trw.load_library()
    n = len(reqs)
    algos = (ctypes.c_int * n)()
    params = (trw._Params * n)()
    srcs = (ctypes.c_void_p * n)()
    ns = (ctypes.c_int64 * n)()
    lens = (ctypes.c_int32 * n)()
    seeds = (ctypes.c_uint64 * n)()
    outs = (ctypes.c_void_p * n)()
    outl = (ctypes.c_void_p * n)()
    keep, results = [], []
    for i, r in enumerate(reqs):
        wps = r.get("walks_per_source", 1)
        ep = r.get("endpoints", False)
        p, k = trw._params(r["algo"], r.get("ppr_stop", 0.2), r.get("n2v_p", 1.0), r.get("n2v_q", 1.0),
                           r.get("schema"), wps, ep, 0, r.get("sampler", trw.SAMPLER_DEFAULT), r.get("max_weight", 0.0))
        src = torch.from_numpy(np.ascontiguousarray(r["sources"], np.int32)).cuda()
        cnt = src.shape[0] * wps
        op = torch.full((cnt,) if ep else (cnt, r["max_len"] + 1), -1, dtype=torch.int32, device="cuda")
        ol = torch.full((cnt,), -1, dtype=torch.int32, device="cuda")
        keep += [k, src]
        algos[i], params[i], srcs[i], ns[i], lens[i] = r["algo"], p, src.data_ptr(), src.shape[0], r["max_len"]
        seeds[i] = r["seed"]
        outs[i], outl[i] = op.data_ptr(), ol.data_ptr()
        results.append((op, ol))
    gc.collect()  # graphs left by earlier tests are freed now, not between the two readings
    torch.cuda.synchronize()
    st_arg = (torch.cuda.current_stream().cuda_stream or 1) if stream == "torch" else None
    free0 = torch.cuda.mem_get_info()[0]
    st = lib.trw_walk_batch_noalloc(G.handle, n, algos, params, srcs, ns, lens, seeds, outs, outl, st_arg)
    free1 = torch.cuda.mem_get_info()[0]
    assert st == 0, lib.trw_last_error()
    torch.cuda.synchronize()
    return results, free0 - free1


def _oracle_results(g, reqs):
    """The oracle's walks of every request (walk i of a request keyed on i)."""
    its = oracle.prepare_its(g.row_ptr, g.weights)
    pmax = oracle.prepare_rej(g.row_ptr, g.weights)
    out = []
    for r in reqs:
        algo = {trw.DEEPWALK: oracle.DEEPWALK, trw.DEEPWALK_WEIGHTED: oracle.DEEPWALK_WEIGHTED, trw.PPR: oracle.PPR,
                trw.NODE2VEC: oracle.NODE2VEC, trw.METAPATH: oracle.METAPATH,
                trw.NODE2VEC_WEIGHTED: oracle.NODE2VEC_WEIGHTED}[r["algo"]]
        sampler = r.get("sampler", trw.SAMPLER_DEFAULT)
        kw = dict(walks_per_source=r.get("walks_per_source", 1), endpoints_only=r.get("endpoints", False),
                  ppr_stop=r.get("ppr_stop", 0.0), n2v_p=r.get("n2v_p", 1.0), n2v_q=r.get("n2v_q", 1.0),
                  max_weight=r.get("max_weight", 0.0))
        if algo == oracle.METAPATH:
            kw.update(labels=g.labels, schema=r["schema"])
        if algo == oracle.DEEPWALK_WEIGHTED:
            if sampler == trw.SAMPLER_DEFAULT:
                kw["alias"] = oracle_alias(12)
            elif sampler == trw.SAMPLER_ITS:
                kw.update(sampler=oracle.SAMPLER_ITS, its=its)
            else:
                kw.update(sampler=oracle.SAMPLER_OREJ, weights=g.weights)
        if algo == oracle.NODE2VEC_WEIGHTED:
            kw.update(weights=g.weights, pmax=pmax)
        res = oracle.walk(g.row_ptr, g.col, algo, r["sources"], r["max_len"], r["seed"], **kw)
        assert res.status == 0, (r["algo"], res.status)
        out.append(res)
    return out


def _same(a_paths, a_lens, b_paths, b_lens):
    assert torch.equal(a_lens, b_lens)
    if a_paths.dim() == 1:
        assert torch.equal(a_paths, b_paths)
    else:
        mask = torch.arange(a_paths.shape[1], device=a_paths.device)[None, :] < a_lens[:, None]
        assert torch.equal(a_paths[mask], b_paths[mask])


def _graph():
    g = rmat_graph(12)
    G = trw.Graph(g.row_ptr, g.col, g.weights, g.labels)
    G.prepare(trw.PREP_ALIAS | trw.PREP_ITS)
    return g, G


def test_noalloc_batch_matches_oracle_and_batch_twice():
    g, G = _graph()
    reqs = _requests(g)
    want = _oracle_results(g, reqs)
    batch = G.walk_batch(reqs)
    torch.cuda.synchronize()
    for _ in range(2):  # the second call reuses the scratch the first one left behind
        got, _ = _call_noalloc(G, reqs)
        for (op, ol), w, b, r in zip(got, want, batch, reqs):
            assert_paths_equal(op.cpu().numpy(), ol.cpu().numpy(), w, endpoints=r.get("endpoints", False))
            _same(b.paths, b.lengths, op, ol)


def test_noalloc_allocates_nothing():
    g, G = _graph()
    reqs = _requests(g)
    want = _oracle_results(g, reqs)
    _call_noalloc(G, reqs)  # the first call on the device may load the module and look up the scratch
    got, used = _call_noalloc(G, reqs)
    assert used == 0, f"the device's free memory fell by {used} bytes during the call"
    # every allocation the library makes now fails as out of memory; this
    # entry point makes none, so it still walks
    trw.fail_allocs(0)
    try:
        got, used = _call_noalloc(G, reqs)
    finally:
        trw.fail_allocs(-1)
    assert used == 0
    for (op, ol), w, r in zip(got, want, reqs):
        assert_paths_equal(op.cpu().numpy(), ol.cpu().numpy(), w, endpoints=r.get("endpoints", False))


def test_noalloc_null_stream():
    g, G = _graph()
    reqs = _requests(g)
    want = _oracle_results(g, reqs)
    for _ in range(2):
        got, _ = _call_noalloc(G, reqs, stream=None)
        for (op, ol), w, r in zip(got, want, reqs):
            assert_paths_equal(op.cpu().numpy(), ol.cpu().numpy(), w, endpoints=r.get("endpoints", False))


def test_noalloc_refuses_oversized_batch():
    g = rmat_graph(12)
    G = trw.Graph(g.row_ptr, g.col, g.weights, g.labels)
    lib = trw.load_library()
    n = 65
    arr = (ctypes.c_void_p * n)()
    st = lib.trw_walk_batch_noalloc(G.handle, n, (ctypes.c_int * n)(), None, arr, (ctypes.c_int64 * n)(),
                                    (ctypes.c_int32 * n)(), (ctypes.c_uint64 * n)(), arr, arr, None)
    assert st == -1
    assert b"no-alloc request table" in lib.trw_last_error()
