"""User-defined walks (include/trw_custom.cuh, GPU only): walk types written
against the header, built into a library, give the oracle's walks for the
same user functions bit for bit."""
import ctypes

import numpy as np
import pytest

import custom_build
import oracle
import paper_2107_11983_gb300 as trw
import synth
from gpu_common import assert_paths_equal, rmat_graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

VP, I32, I64, U32, U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    trw.load_library()
    so = custom_build.build(str(tmp_path_factory.mktemp("custom")))
    L = ctypes.CDLL(so)
    L.tw_naive.argtypes = [VP, VP, I64, I32, I32, U64, U32, VP, VP, VP]
    L.tw_stop_on_multiple.argtypes = [VP, VP, I64, I32, U64, I32, VP, VP, VP]
    L.tw_node2vec.argtypes = [VP, VP, I64, I32, U64, I32, U32, VP, VP, VP]
    L.tw_endpoint_weight.argtypes = [VP, VP, I64, I32, I32, U64, VP, VP, VP]
    return L


@pytest.fixture(scope="module")
def graph():
    g = rmat_graph(12)
    return g, trw.Graph(g.row_ptr, g.col, g.weights)


def buffers(n, L):
    return (torch.empty((n, L + 1), dtype=torch.int32, device="cuda"),
            torch.empty(n, dtype=torch.int32, device="cuda"))


def check(st, paths, lengths, moves, want):
    assert st == 0, st
    torch.cuda.synchronize()
    assert_paths_equal(paths.cpu().numpy(), lengths.cpu().numpy(), want)
    assert moves.value == int((want.lengths - 1).sum())


def test_naive_with_offsets(lib, graph):
    g, G = graph
    src = synth.sources(3000, g.nv, seed=1)
    d = torch.from_numpy(src).cuda()
    p, l = buffers(6000, 40)
    m = I64(0)
    st = lib.tw_naive(G.handle, d.data_ptr(), 3000, 2, 40, 77, 1234, p.data_ptr(), l.data_ptr(), ctypes.byref(m))
    want = oracle.walk_custom(g.row_ptr, g.col, src, 40, 77, sampler=oracle.NAIVE_SAMPLER, walks_per_source=2,
                              walk_offset=1234)
    check(st, p, l, m, want)
    dw = oracle.walk(g.row_ptr, g.col, oracle.DEEPWALK, src, 40, 77, walks_per_source=2, walk_offset=1234)
    assert np.array_equal(want.lengths, dw.lengths)  # the restatement is DeepWalk


def test_update_ends_walks(lib, graph):
    g, G = graph
    src = synth.vertex_sources(g.nv)
    d = torch.from_numpy(src).cuda()
    p, l = buffers(g.nv, 60)
    m = I64(0)
    st = lib.tw_stop_on_multiple(G.handle, d.data_ptr(), g.nv, 60, 5, 7, p.data_ptr(), l.data_ptr(), ctypes.byref(m))
    want = oracle.walk_custom(g.row_ptr, g.col, src, 60, 5, sampler=oracle.NAIVE_SAMPLER,
                              update=lambda w, ln, cur, prev, dst, e: cur % 7 == 0)
    check(st, p, l, m, want)


@pytest.mark.parametrize("weighted", [0, 1], ids=["node2vec", "weighted-node2vec"])
def test_node2vec_in_ten_lines(lib, graph, weighted):
    g, G = graph
    src = np.concatenate([synth.vertex_sources(g.nv), synth.sources(500, g.nv, seed=3)])
    d = torch.from_numpy(src).cuda()
    p, l = buffers(src.shape[0], 30)
    m = I64(0)
    bound = 100 * 65536
    st = lib.tw_node2vec(G.handle, d.data_ptr(), src.shape[0], 30, 9, weighted, bound, p.data_ptr(), l.data_ptr(),
                         ctypes.byref(m))
    adj = [set(g.col[g.row_ptr[v]:g.row_ptr[v + 1]].tolist()) for v in range(g.nv)]
    Wq = np.minimum(np.rint(g.weights.astype(np.float64) * 65536), 2 ** 32 - 1).astype(np.int64)

    def weight(w, ln, cur, prev, dst, e):
        c = 4 if ln == 0 else (4 if dst == prev else (2 if dst in adj[prev] else 1))
        return min(2 ** 32 - 1, c * int(Wq[e])) if weighted else c

    want = oracle.walk_custom(g.row_ptr, g.col, src, 30, 9, sampler=oracle.OREJ_SAMPLER, weight=weight,
                              max_weight=4 * bound if weighted else 4)
    check(st, p, l, m, want)
    if not weighted:  # the ten lines are the built-in Node2Vec (a = 0.5, b = 2)
        out = G.walk(trw.NODE2VEC, d, 30, seed=9, n2v_p=0.5, n2v_q=2.0)
        torch.cuda.synchronize()
        assert np.array_equal(out.lengths.cpu().numpy(), want.lengths)


def test_endpoint_weight_and_errors(lib, graph):
    g, G = graph
    src = synth.sources(2000, g.nv, seed=6)
    d = torch.from_numpy(src).cuda()
    p, l = buffers(4000, 25)
    m = I64(0)
    st = lib.tw_endpoint_weight(G.handle, d.data_ptr(), 2000, 2, 25, 4, p.data_ptr(), l.data_ptr(), ctypes.byref(m))
    want = oracle.walk_custom(g.row_ptr, g.col, src, 25, 4, sampler=oracle.OREJ_SAMPLER,
                              weight=lambda w, ln, cur, prev, dst, e: 1 + 3 * ((cur + 2 * dst) % 3), max_weight=7,
                              walks_per_source=2)
    check(st, p, l, m, want)
    bad = torch.from_numpy(np.array([0, g.nv + 5], np.int32)).cuda()
    st = lib.tw_naive(G.handle, bad.data_ptr(), 2, 1, 10, 1, 0, p.data_ptr(), l.data_ptr(), ctypes.byref(m))
    assert st == -1
    st = lib.tw_naive(G.handle, d.data_ptr(), 2000, 1, 10, 1, 2 ** 32 - 10, p.data_ptr(), l.data_ptr(),
                      ctypes.byref(m))
    assert st == -1  # walk indices past 2^32
    st = lib.tw_naive(None, d.data_ptr(), 2000, 1, 10, 1, 0, p.data_ptr(), l.data_ptr(), ctypes.byref(m))
    assert st == -1
