"""Serving loop (GPU only): requests of different algorithms and sizes join a
running persistent kernel, and every result is bit-identical to the oracle,
alone or in the mix."""
import time

import numpy as np
import pytest

import paper_2107_11983_gb300 as trw
import synth
from gpu_common import assert_paths_equal, oracle_alias, oracle_walk, rmat_graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SCALE = 12
SCHEMA = np.array([1, 3, 0, 4, 2], np.uint8)


@pytest.fixture
def server_factory():
    made = []

    def make(G, **kw):
        S = trw.Server(G, **kw)
        made.append(S)
        return S

    yield make
    for S in made:
        S.close()


@pytest.fixture(scope="module")
def served():
    g = rmat_graph(SCALE)
    G = trw.Graph(g.row_ptr, g.col, g.weights, g.labels)
    G.prepare()
    return g, G


def make_request(g, i, rng):
    kind = i % 5
    n = int(rng.integers(1, 3000))
    src = synth.sources(n, g.nv, seed=100 + i)
    if kind == 0:
        return dict(algo=trw.PPR, sources=src[:1], walks_per_source=n, max_len=1000, seed=i, ppr_stop=0.2,
                    endpoints=True)
    if kind == 1:
        return dict(algo=trw.DEEPWALK, sources=src, max_len=80, seed=i)
    if kind == 2:
        return dict(algo=trw.DEEPWALK_WEIGHTED, sources=src, max_len=80, seed=i)
    if kind == 3:
        return dict(algo=trw.NODE2VEC, sources=src, max_len=80, seed=i, n2v_p=0.5, n2v_q=2.0)
    return dict(algo=trw.METAPATH, sources=src, max_len=60, seed=i, schema=SCHEMA)


def submit(S, r):
    n = r["sources"].shape[0] * r.get("walks_per_source", 1)
    shape = (n,) if r.get("endpoints") else (n, r["max_len"] + 1)
    op = torch.full(shape, -1, dtype=torch.int32, device="cuda")
    ol = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    kw = {k: r[k] for k in ("ppr_stop", "n2v_p", "n2v_q", "schema", "walks_per_source", "endpoints") if k in r}
    rid = S.submit(r["algo"], r["sources"], r["max_len"], r["seed"], op, ol, **kw)
    return rid, op, ol


def check(g, r, op, ol):
    kw = {k: r[k] for k in ("ppr_stop", "n2v_p", "n2v_q", "schema", "walks_per_source") if k in r}
    want = oracle_walk(g, r["algo"], r["sources"], r["max_len"], r["seed"],
                       alias=oracle_alias(SCALE) if r["algo"] == trw.DEEPWALK_WEIGHTED else None,
                       endpoints_only=r.get("endpoints", False), **kw)
    assert_paths_equal(op.cpu().numpy(), ol.cpu().numpy(), want, endpoints=r.get("endpoints", False))


def wait(S, rid, timeout=60.0):
    t = time.time()
    while S.poll(rid) == trw.PENDING:
        assert time.time() - t < timeout, f"request {rid} did not finish"
        time.sleep(0.0005)


def test_serve_mix_matches_oracle(served, server_factory):
    g, G = served
    S = server_factory(G, max_requests=64)
    rng = np.random.default_rng(0)
    reqs = [make_request(g, i, rng) for i in range(40)]
    live = []
    for r in reqs:  # submitted back to back: later requests join the running kernel
        live.append((r,) + submit(S, r))
    for r, rid, op, ol in live:
        wait(S, rid)
        check(g, r, op, ol)


def test_serve_same_alone_and_in_mix(served, server_factory):
    g, G = served
    rng = np.random.default_rng(1)
    reqs = [make_request(g, i, rng) for i in range(10)]
    S = server_factory(G, max_requests=32)
    alone = []
    for r in reqs:
        rid, op, ol = submit(S, r)
        wait(S, rid)
        alone.append((op.clone(), ol.clone()))
    # now the same requests overlapped with a large background request
    big = dict(algo=trw.NODE2VEC, sources=synth.vertex_sources(g.nv), max_len=80, seed=999, n2v_p=0.5, n2v_q=2.0)
    brid, bop, bol = submit(S, big)
    mixed = [submit(S, r) for r in reqs]
    for (rid, op, ol), (aop, aol) in zip(mixed, alone):
        wait(S, rid)
        assert torch.equal(ol, aol)
        if op.dim() == 1:
            assert torch.equal(op, aop)
        else:
            mask = torch.arange(op.shape[1], device="cuda")[None, :] < ol[:, None]
            assert torch.equal(op[mask], aop[mask])
    wait(S, brid)
    check(g, big, bop, bol)


def test_serve_admission_and_ids(served, server_factory):
    g, G = served
    S = server_factory(G, max_requests=4, max_inflight_walks=5000)
    r = dict(algo=trw.DEEPWALK, sources=synth.sources(3000, g.nv, seed=5), max_len=80, seed=1)
    rid, op, ol = submit(S, r)
    # too many walks in flight -> busy, nothing queued
    with pytest.raises(trw.TRWError) as e:
        submit(S, dict(r, sources=synth.sources(2500, g.nv, seed=6)))
    assert e.value.status == -7
    wait(S, rid)
    check(g, r, op, ol)
    with pytest.raises(trw.TRWError) as e:
        S.poll(rid)  # already collected
    assert e.value.status == -8
    with pytest.raises(trw.TRWError) as e:
        S.poll(12345)
    assert e.value.status == -8
    # more requests than slots, in sequence: slots and source ranges are reused
    for i in range(12):
        rr = dict(algo=trw.PPR, sources=synth.sources(1, g.nv, seed=i), walks_per_source=1000, max_len=1000,
                  seed=i, ppr_stop=0.2, endpoints=True)
        rid, op, ol = submit(S, rr)
        wait(S, rid)
        check(g, rr, op, ol)
    # invalid requests are refused at submit
    with pytest.raises(trw.TRWError) as e:
        submit(S, dict(r, sources=np.array([g.nv], np.int32)))
    assert e.value.status == -1


def test_serve_warp_cooperative_rows(served, server_factory):
    g, G = served
    old = G.tuning()
    G.set_tuning(coop_degree=1, search_degree=33)  # MetaPath scans and neighbour checks go to the warp
    try:
        S = server_factory(G, max_requests=16)
        rng = np.random.default_rng(5)
        reqs = [make_request(g, i, rng) for i in range(10)]
        live = [(r,) + submit(S, r) for r in reqs]
        for r, rid, op, ol in live:
            wait(S, rid)
            check(g, r, op, ol)
    finally:
        G.set_tuning(**old)


def test_serve_relaunch_after_idle(served, server_factory):
    g, G = served
    S = server_factory(G, max_requests=8, idle_timeout_us=200)
    for i in range(3):
        r = dict(algo=trw.DEEPWALK_WEIGHTED, sources=synth.sources(500, g.nv, seed=40 + i), max_len=30, seed=i)
        rid, op, ol = submit(S, r)
        wait(S, rid)
        check(g, r, op, ol)
        time.sleep(0.05)  # longer than the idle timeout: the resident kernel exits
    S.drain(10000)


def test_serve_device_source_check_and_reap(served, server_factory):
    """Device sources are checked at submit: an out-of-range one is refused
    with ERR_INVALID and nothing written, while the requests around it run;
    reap collects every finished request in one call."""
    g, G = served
    S = server_factory(G, max_requests=32)
    rng = np.random.default_rng(9)
    reqs = [make_request(g, i, rng) for i in range(12)]
    bad_src = torch.from_numpy(synth.sources(2000, g.nv, seed=77)).cuda()
    bad_src[1234] = g.nv
    bad = dict(algo=trw.DEEPWALK, sources=bad_src, max_len=40, seed=3)
    live = {}
    for i, r in enumerate(reqs):
        rr = dict(r, sources=torch.from_numpy(r["sources"]).cuda())
        rid, op, ol = submit(S, rr)
        live[rid] = (r, op, ol)
        if i == 5:
            bop = torch.full((2000, 41), -1, dtype=torch.int32, device="cuda")
            bol = torch.full((2000,), -1, dtype=torch.int32, device="cuda")
            with pytest.raises(trw.TRWError) as e:
                S.submit(bad["algo"], bad["sources"], bad["max_len"], bad["seed"], bop, bol)
            assert e.value.status == -1
    statuses = {}
    t = time.time()
    while len(statuses) < len(live):
        for rid, st in S.reap(max_requests=4):
            assert rid not in statuses
            statuses[rid] = st
        assert time.time() - t < 60, "requests did not finish"
        time.sleep(0.0005)
    torch.cuda.synchronize()
    assert bool((bol == -1).all()) and bool((bop == -1).all())
    for rid, (r, op, ol) in live.items():
        assert statuses[rid] == 0
        check(g, r, op, ol)
    assert S.reap() == []
    with pytest.raises(trw.TRWError) as e:
        S.poll(next(iter(live)))  # already collected by reap
    assert e.value.status == -8


def test_serve_small_device_sources_checked_on_device(served, server_factory):
    """A small request's device sources are range-checked when the server
    admits it: one out of range completes that request with ERR_INVALID at
    reap, writes nothing, and the requests around it match the oracle."""
    g, G = served
    S = server_factory(G, max_requests=32)
    rng = np.random.default_rng(21)
    reqs = [make_request(g, i, rng) for i in range(8)]
    bad_src = torch.from_numpy(synth.sources(500, g.nv, seed=78)).cuda()
    bad_src[321] = g.nv + 5
    neg_src = torch.from_numpy(synth.sources(3, g.nv, seed=79)).cuda()
    neg_src[2] = -1
    live, bad_ids = {}, {}
    for i, r in enumerate(reqs):
        rid, op, ol = submit(S, dict(r, sources=torch.from_numpy(r["sources"]).cuda()))
        live[rid] = (r, op, ol)
        if i in (2, 5):
            src = bad_src if i == 2 else neg_src
            n = int(src.shape[0])
            bop = torch.full((n, 41), -1, dtype=torch.int32, device="cuda")
            bol = torch.full((n,), -1, dtype=torch.int32, device="cuda")
            bad_ids[S.submit(trw.DEEPWALK, src, 40, 3, bop, bol)] = (bop, bol)
    statuses = {}
    t = time.time()
    while len(statuses) < len(live) + len(bad_ids):
        for rid, st in S.reap():
            statuses[rid] = st
        assert time.time() - t < 60, "requests did not finish"
        time.sleep(0.0005)
    torch.cuda.synchronize()
    for rid, (bop, bol) in bad_ids.items():
        assert statuses[rid] == -1
        assert bool((bol == -1).all()) and bool((bop == -1).all())
    for rid, (r, op, ol) in live.items():
        assert statuses[rid] == 0
        check(g, r, op, ol)


def test_serve_trace_timeline(served, server_factory):
    """Every served request carries a device timeline: admitted, started and
    finished, in that order."""
    g, G = served
    S = server_factory(G, max_requests=16)
    rng = np.random.default_rng(11)
    reqs = [make_request(g, i, rng) for i in range(6)]
    live = [(r,) + submit(S, r) for r in reqs]
    for r, rid, op, ol in live:
        wait(S, rid)
        check(g, r, op, ol)
        t = S.trace(rid)
        assert 0 < t["admit_ns"] <= t["first_ns"] <= t["done_ns"], t
    with pytest.raises(trw.TRWError) as e:
        S.trace(10 ** 6)
    assert e.value.status == -8


@pytest.mark.parametrize("n", [300, 3000], ids=["checked-on-device", "checked-on-host"])
def test_serve_waits_for_the_callers_stream(served, server_factory, n):
    """A request whose device sources are still being written on the caller's
    stream (a long-running kernel ahead of the write) runs on the written
    sources: the submit publishes it only after that stream's work, whether
    the dispatcher or the host range-checks the sources.  Requests submitted
    while the stream is idle publish straight away (the other serve tests)."""
    g, G = served
    S = server_factory(G)
    want_src = synth.sources(n, g.nv, seed=77)
    r = dict(algo=trw.DEEPWALK, sources=want_src, max_len=40, seed=5)
    src = torch.full((n,), g.nv + 7, dtype=torch.int32, device="cuda")  # out of range until written
    good = torch.from_numpy(want_src).cuda()
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        torch.cuda._sleep(50_000_000)  # tens of milliseconds of device time before the write
        src.copy_(good)
        op = torch.full((n, 41), -1, dtype=torch.int32, device="cuda")
        ol = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        assert not stream.query(), "the caller's stream finished before the submit: nothing to order"
        rid = S.submit(trw.DEEPWALK, src, 40, 5, op, ol)
    wait(S, rid)
    check(g, r, op, ol)


def test_serve_mixes_ordered_and_direct_publication(served, server_factory):
    """Requests published through the copy stream (the caller's stream still
    busy) and straight into mapped memory (an idle stream) interleave without
    a request lost, admitted twice or out of order: every result is the
    oracle's."""
    g, G = served
    S = server_factory(G)
    rng = np.random.default_rng(9)
    busy = torch.cuda.Stream()
    idle = torch.cuda.Stream()
    reqs, out = [], []
    for i in range(12):
        n = int(rng.integers(50, 400))
        src_h = synth.sources(n, g.nv, seed=300 + i)
        r = dict(algo=trw.DEEPWALK if i % 2 else trw.PPR, sources=src_h, max_len=30, seed=40 + i, ppr_stop=0.2)
        src = torch.from_numpy(src_h).cuda()
        op = torch.full((n, 31), -1, dtype=torch.int32, device="cuda")
        ol = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        if i % 4 == 0:
            # a request behind device work on its stream: published through the copy stream
            with torch.cuda.stream(busy):
                torch.cuda._sleep(5_000_000)
                rid = S.submit(r["algo"], src, 30, r["seed"], op, ol, ppr_stop=0.2)
        else:
            with torch.cuda.stream(idle):
                rid = S.submit(r["algo"], src, 30, r["seed"], op, ol, ppr_stop=0.2)
        reqs.append(r)
        out.append((rid, op, ol))
    assert [rid for rid, _, _ in out] == list(range(out[0][0], out[0][0] + 12))
    for r, (rid, op, ol) in zip(reqs, out):
        wait(S, rid)
        check(g, r, op, ol)


def test_serve_two_ordering_calls_before_a_submit(served, server_factory):
    """Through the C entry points: ordering after stream A, then after stream
    B, then one submit.  The request waits for both streams' earlier work,
    not only the last one's: its sources are written on A behind a long
    kernel, while B has little to do."""
    import ctypes
    g, G = served
    S = server_factory(G)
    lib = trw.load_library()
    n = 200
    want_src = synth.sources(n, g.nv, seed=88)
    src = torch.full((n,), g.nv + 3, dtype=torch.int32, device="cuda")  # out of range until written
    good = torch.from_numpy(want_src).cuda()
    op = torch.full((n, 31), -1, dtype=torch.int32, device="cuda")
    ol = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    a, b = torch.cuda.Stream(), torch.cuda.Stream()
    with torch.cuda.stream(a):
        torch.cuda._sleep(50_000_000)
        src.copy_(good)
    with torch.cuda.stream(b):
        torch.cuda._sleep(1_000_000)
    assert not a.query() and not b.query()
    assert lib.trw_serve_order_after(S._h, a.cuda_stream) == 0
    assert lib.trw_serve_order_after(S._h, b.cuda_stream) == 0
    p, keep = trw._params(trw.DEEPWALK, 0.2, 1.0, 1.0, None, 1, False, 0, trw.SAMPLER_DEFAULT, 0.0)
    rid = ctypes.c_uint64(0)
    assert lib.trw_serve_submit(S._h, trw.DEEPWALK, ctypes.byref(p), src.data_ptr(), n, 30, 7, op.data_ptr(),
                                ol.data_ptr(), ctypes.byref(rid)) == 0
    wait(S, rid.value)
    check(g, dict(algo=trw.DEEPWALK, sources=want_src, max_len=30, seed=7), op, ol)
