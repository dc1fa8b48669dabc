"""Pins of the oracle to things other than itself.

Each pin takes a bound oracle library (the real one, or a copy with a planted
mistake) and raises AssertionError when the oracle disagrees with what the
paper or the mathematics fixes:

  * published known-answer vectors of Philox4x32-10;
  * closed forms of the fixed-point conventions (thresholds, quantisation);
  * the exact law implied by every alias table (exact rationals);
  * exact path laws on tiny graphs, enumerated by brute force from the
    transition rules of Section 2.2 (first order, Node2Vec Eq. 1 over
    (prev, cur) pairs, MetaPath's label filter), tested by chi-square;
  * the PPR end-vertex law by a linear solve of the absorbing chain, and the
    geometric length law (mean 5 vertices at stop 0.2, Section 6.2);
  * the O-REJ expected number of trials d * p* / sum(p) (Section 2.3);
  * the sector model of the statistics (distinct 32-byte sectors a move
    reads in the device layout, and the output bytes) against hand counts
    on tiny graphs;
  * special cases that must reduce exactly to NAIVE sampling;
  * weighted DeepWalk under ITS, REJ and O-REJ: the first move of every walk
    recomputed independently (numpy prefix sums and searchsorted for ITS,
    the dart sequence with the cross-multiplied acceptance test for REJ and
    O-REJ), path laws by chi-square, the expected trials d * p* / sum(p)
    on a graph whose rows share one weight multiset, and the acceptance
    threshold by its counting definition.
"""
from __future__ import annotations

import itertools
import os
from collections import Counter
from fractions import Fraction

import numpy as np
from scipy import stats as sst

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))
TWO32 = 1 << 32

# --------------------------------------------------------------- tiny graphs

# A directed graph with a dead end (5) and asymmetric adjacency, so that
# IsNeighbor's direction matters.
DIR_EDGES = [(0, 1), (0, 2), (0, 3), (1, 0), (1, 2), (1, 4), (2, 0), (2, 3), (2, 5),
             (3, 1), (3, 4), (3, 5), (3, 6), (4, 0), (4, 3), (6, 0), (6, 2)]
DIR_NV = 7
# Distinct positive weights for the weighted walk, by edge.
DIR_WEIGHTS = {e: float(w) for e, w in zip(DIR_EDGES, [1, 2, 7, 3, 1.5, 4, 2.25, 9, 1, 5, 1, 2, 3.5, 6, 1, 1, 8])}
# Labels in {0,1,2} for MetaPath.
DIR_LABELS = {e: l for e, l in zip(DIR_EDGES, [0, 1, 0, 1, 1, 0, 2, 0, 1, 0, 1, 1, 0, 1, 0, 0, 1])}

N_LAW = 200_000


def dir_graph():
    g = synth.from_edges(DIR_NV, DIR_EDGES, symmetric=False)
    w = np.array([DIR_WEIGHTS[(v, int(c))] for v in range(DIR_NV)
                  for c in g.col[g.row_ptr[v]:g.row_ptr[v + 1]]], dtype=np.float32)
    lab = np.array([DIR_LABELS[(v, int(c))] for v in range(DIR_NV)
                    for c in g.col[g.row_ptr[v]:g.row_ptr[v + 1]]], dtype=np.uint8)
    g.weights, g.labels = w, lab
    return g


def nbrs(g, v):
    return [int(c) for c in g.col[g.row_ptr[v]:g.row_ptr[v + 1]]]


# ------------------------------------------------------------------ helpers

def chi2_pvalue(counts: Counter, probs: dict, n: int) -> float:
    """Chi-square goodness of fit; cells with expected count < 5 are pooled.
    An outcome of probability zero that was observed gives p = 0."""
    for k, c in counts.items():
        if c > 0 and probs.get(k, 0.0) == 0.0:
            return 0.0
    obs, exp, pool_o, pool_e = [], [], 0.0, 0.0
    for k, p in probs.items():
        e = p * n
        if e < 5:
            pool_o += counts.get(k, 0)
            pool_e += e
        else:
            obs.append(counts.get(k, 0))
            exp.append(e)
    if pool_e > 0:
        obs.append(pool_o)
        exp.append(pool_e)
    obs = np.array(obs, dtype=np.float64)
    exp = np.array(exp, dtype=np.float64)
    exp *= obs.sum() / exp.sum()
    if len(obs) < 2:
        return 1.0
    return float(sst.chisquare(obs, exp).pvalue)


def path_counts(res) -> Counter:
    c = Counter()
    for row, ln in zip(res.paths, res.lengths):
        c[tuple(int(x) for x in row[:ln])] += 1
    return c


def enumerate_paths(src: int, max_len: int, step_law) -> dict:
    """Exact law over whole paths: step_law(path) -> {next: prob} ({} = stop)."""
    out = {}

    def rec(path, p):
        if len(path) - 1 == max_len:
            out[tuple(path)] = out.get(tuple(path), 0.0) + p
            return
        law = step_law(path)
        if not law:
            out[tuple(path)] = out.get(tuple(path), 0.0) + p
            return
        for nxt, q in law.items():
            if q > 0:
                rec(path + [nxt], p * q)

    rec([src], 1.0)
    return out


# ------------------------------------------------------------------- pins

def pin_philox_kat(lib=None):
    path = os.path.join(HERE, "golden", "philox4x32_10_kat.txt")
    n = 0
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        w = [int(x, 16) for x in line.split()]
        got = oracle.philox4x32_10(w[0:4], w[4:6], lib=lib)
        assert list(map(int, got)) == w[6:10], f"Philox KAT mismatch for {line}"
        n += 1
    assert n == 3


def pin_fixed_point(lib=None):
    # floor(t * 2^32) as an exact rational of the double t.
    for t in [0.2, 0.5, 0.25, 1 / 3, 0.7, 1e-9, 0.999999999]:
        want = (Fraction(t) * TWO32).numerator // (Fraction(t) * TWO32).denominator
        assert oracle.threshold(t, lib=lib) == want, t
    assert oracle.threshold(0.2, lib=lib) == 858993459
    assert oracle.threshold(0.0, lib=lib) == 0
    assert oracle.threshold(1.0, lib=lib) == TWO32
    # round-half-even(w * 2^16): ties of exactly representable fp32 values
    assert oracle.quantize_weight(1.0, lib=lib) == 65536
    assert oracle.quantize_weight(1.5 / 65536, lib=lib) == 2
    assert oracle.quantize_weight(2.5 / 65536, lib=lib) == 2
    assert oracle.quantize_weight(3.5 / 65536, lib=lib) == 4
    assert oracle.quantize_weight(0.75 / 65536, lib=lib) == 1
    assert oracle.quantize_weight(0.25 / 65536, lib=lib) == 0
    assert oracle.quantize_weight(99.99999, lib=lib) == round(float(np.float32(99.99999)) * 65536)
    assert oracle.quantize_weight(1e30, lib=lib) == TWO32 - 1
    assert oracle.quantize_weight(-1.0, lib=lib) == -1
    assert oracle.quantize_weight(float("nan"), lib=lib) == -1
    assert oracle.quantize_weight(float("inf"), lib=lib) == -1


def _alias_rows():
    rng = np.random.default_rng(7)
    rows = [[5], [1, 1], [3, 3, 3, 3], [1, 2, 3, 4], [0, 7, 0, 1], [0, 0, 5], [2 ** 32 - 1, 1, 1],
            [65536 * 99, 65536, 65536 * 50, 65537]]
    rows += [list(rng.integers(65536, 6553600, size=d)) for d in (5, 17, 64, 300)]
    rows += [list(rng.integers(0, 4, size=50))]
    return rows


def pin_alias_law(lib=None):
    """The law implied by the tables is W_j / S within 2^-32 per bucket:
    sum_j |P_j - W_j/S| <= 2 * 2^-32 (each bucket's floor moves < 2^-32 / d
    of mass between its two elements)."""
    for W in _alias_rows():
        d = len(W)
        H, A1, A2, dead = oracle.alias_build(W, lib=lib)
        S = sum(int(x) for x in W)
        assert dead == (1 if S == 0 else 0)
        if S == 0:
            continue
        mass = [Fraction(0)] * d
        for b in range(d):
            h = int(H[b])
            assert 0 <= h <= TWO32
            assert int(A1[b]) == b, "first element of bucket b is b"
            if h < TWO32:
                assert 0 <= int(A2[b]) < d
                mass[int(A2[b])] += Fraction(TWO32 - h, TWO32 * d)
            mass[b] += Fraction(h, TWO32 * d)
        err = sum(abs(mass[j] - Fraction(int(W[j]), S)) for j in range(d))
        assert err <= Fraction(2, TWO32), (W, float(err))
        for j in range(d):
            if int(W[j]) == 0:
                assert mass[j] == 0, "a zero-weight edge is never picked"


def _dir_alias(g, lib):
    return oracle.prepare_alias(g.row_ptr, g.weights, lib=lib)


def pin_law_deepwalk(lib=None):
    g = dir_graph()
    res = oracle.walk(g.row_ptr, g.col, oracle.DEEPWALK, [0], 3, seed=11, walks_per_source=N_LAW, lib=lib)
    assert res.status == 0

    def law(path):
        nb = nbrs(g, path[-1])
        return {c: 1.0 / len(nb) for c in nb}

    p = chi2_pvalue(path_counts(res), enumerate_paths(0, 3, law), N_LAW)
    assert p > 1e-3, p


def pin_law_alias(lib=None):
    g = dir_graph()
    al = _dir_alias(g, lib)
    res = oracle.walk(g.row_ptr, g.col, oracle.DEEPWALK_WEIGHTED, [0], 3, seed=12, walks_per_source=N_LAW,
                      alias=al, lib=lib)
    assert res.status == 0

    def law(path):
        v = path[-1]
        nb = nbrs(g, v)
        ws = [DIR_WEIGHTS[(v, c)] for c in nb]
        return {c: w / sum(ws) for c, w in zip(nb, ws)}

    p = chi2_pvalue(path_counts(res), enumerate_paths(0, 3, law), N_LAW)
    assert p > 1e-3, p


def node2vec_step_law(g, path, p_ret, q_io):
    """Eq. 1 with O-REJ's fixed-point acceptance T_k = floor(w_k / p* * 2^32):
    candidate c is taken with probability proportional to T_class(c)."""
    v = path[-1]
    nb = nbrs(g, v)
    if not nb:
        return {}
    if len(path) == 1:
        return {c: 1.0 / len(nb) for c in nb}
    u = path[-2]
    w_ret, w_nb, w_far = 1.0 / p_ret, 1.0, 1.0 / q_io
    pstar = max(w_ret, w_nb, w_far)
    T = {k: (Fraction(x / pstar) * TWO32).__floor__() for k, x in (("r", w_ret), ("n", w_nb), ("f", w_far))}
    nu = set(nbrs(g, u))
    t = {c: T["r"] if c == u else (T["n"] if c in nu else T["f"]) for c in nb}
    tot = sum(t.values())
    return {c: t[c] / tot for c in nb}


def pin_law_node2vec(lib=None):
    g = dir_graph()
    for (pp, qq, seed) in [(0.5, 2.0, 13), (2.0, 0.5, 14), (0.3, 0.7, 15)]:
        res = oracle.walk(g.row_ptr, g.col, oracle.NODE2VEC, [0], 3, seed=seed, walks_per_source=N_LAW,
                          n2v_p=pp, n2v_q=qq, lib=lib)
        assert res.status == 0
        law = enumerate_paths(0, 3, lambda path: node2vec_step_law(g, path, pp, qq))
        p = chi2_pvalue(path_counts(res), law, N_LAW)
        assert p > 1e-3, (pp, qq, p)


def pin_law_metapath(lib=None):
    g = dir_graph()
    schema = [0, 1, 1]
    res = oracle.walk(g.row_ptr, g.col, oracle.METAPATH, [0, 3], 4, seed=16, walks_per_source=N_LAW // 2,
                      labels=g.labels, schema=schema, lib=lib)
    assert res.status == 0

    def law(path):
        v = path[-1]
        s = len(path) - 1
        h = schema[s % len(schema)]
        ok = [c for c in nbrs(g, v) if DIR_LABELS[(v, c)] == h]
        return {c: 1.0 / len(ok) for c in ok}

    for src, lo in ((0, 0), (3, N_LAW // 2)):
        sub = type(res)(res.paths[lo:lo + N_LAW // 2], res.lengths[lo:lo + N_LAW // 2], {}, 0)
        p = chi2_pvalue(path_counts(sub), enumerate_paths(src, 4, law), N_LAW // 2)
        assert p > 1e-3, (src, p)


def ppr_end_law(g, src, alpha):
    """End-vertex law of a walk that stops with probability alpha before each
    move and at dead ends: pi = e_s (I - M)^-1 diag(sigma), M = diag(1-sigma) P."""
    nv = g.nv
    P = np.zeros((nv, nv))
    sigma = np.ones(nv)
    for v in range(nv):
        nb = nbrs(g, v)
        if nb:
            sigma[v] = alpha
            for c in nb:
                P[v, c] = 1.0 / len(nb)
    M = np.diag(1 - sigma) @ P
    e = np.zeros(nv)
    e[src] = 1.0
    pi = np.linalg.solve((np.eye(nv) - M).T, e) * sigma
    return {v: float(pi[v]) for v in range(nv)}


def pin_ppr(lib=None):
    g = dir_graph()
    n = N_LAW
    res = oracle.walk(g.row_ptr, g.col, oracle.PPR, [1], 1000, seed=17, walks_per_source=n, ppr_stop=0.2,
                      endpoints_only=True, lib=lib)
    assert res.status == 0
    p = chi2_pvalue(Counter(int(x) for x in res.paths), ppr_end_law(g, 1, 0.2), n)
    assert p > 1e-3, p
    # Geometric lengths on a graph without dead ends: P(moves = k) = 0.8^k * 0.2,
    # so E|Q| = 5 vertices (Section 6.2).
    k4 = synth.from_edges(4, [(a, b) for a in range(4) for b in range(4) if a != b])
    res = oracle.walk(k4.row_ptr, k4.col, oracle.PPR, [0], 1000, seed=18, walks_per_source=n, ppr_stop=0.2,
                      lib=lib)
    assert res.status == 0
    moves = res.lengths.astype(np.int64) - 1
    law = {k: 0.8 ** k * 0.2 for k in range(200)}
    p = chi2_pvalue(Counter(int(m) for m in moves), law, n)
    assert p > 1e-3, p
    mean_q = res.lengths.mean()
    assert abs(mean_q - 5.0) < 6 * np.sqrt(20.0 / n), mean_q  # var of moves = 0.8/0.04 = 20


def pin_rejection_trials(lib=None):
    """Mean O-REJ trials per step equal d * 2^32 / sum_c T_class(c): the
    fixed-point form of E = d * p* / sum(p) (Section 2.3)."""
    g = dir_graph()
    pp, qq = 0.5, 2.0
    n = N_LAW
    res = oracle.walk(g.row_ptr, g.col, oracle.NODE2VEC, [0], 2, seed=19, walks_per_source=n, n2v_p=pp,
                      n2v_q=qq, lib=lib)
    assert res.status == 0
    n0 = nbrs(g, 0)
    mean = 1.0
    second = 0.0
    for v1 in n0:
        law = node2vec_step_law(g, [0, v1], pp, qq)
        if not law:
            continue
        d = len(nbrs(g, v1))
        w_ret, w_nb, w_far = 1.0 / pp, 1.0, 1.0 / qq
        pstar = max(w_ret, w_nb, w_far)
        T = {"r": (Fraction(w_ret / pstar) * TWO32).__floor__(), "n": (Fraction(w_nb / pstar) * TWO32).__floor__(),
             "f": (Fraction(w_far / pstar) * TWO32).__floor__()}
        nu = set(nbrs(g, 0))
        acc = sum((T["r"] if c == 0 else (T["n"] if c in nu else T["f"])) for c in nbrs(g, v1)) / (d * TWO32)
        e = 1.0 / acc
        var = (1 - acc) / acc ** 2
        mean += e / len(n0)
        second += (var + e * e) / len(n0)
    var_tot = second - (mean - 1.0) ** 2
    got = res.stats["attempts"] / n
    assert abs(got - mean) < 6 * np.sqrt(var_tot / n), (got, mean)


def small_rmat():
    g = synth.rmat(10, seed=5)
    g.weights = synth.edge_weights(g, seed=5)
    g.labels = synth.edge_labels(g, seed=5, nlabels=5)
    return g


def pin_reductions(lib=None):
    """Cases that must be bit-identical to NAIVE DeepWalk (same draw, same index)."""
    g = small_rmat()
    src = synth.vertex_sources(g.nv)
    L = 20
    base = oracle.walk(g.row_ptr, g.col, oracle.DEEPWALK, src, L, seed=3, lib=lib)
    assert base.status == 0

    def same(res, what):
        assert res.status == 0, what
        assert np.array_equal(res.lengths, base.lengths), what
        for i in range(g.nv):
            ln = base.lengths[i]
            assert np.array_equal(res.paths[i, :ln], base.paths[i, :ln]), (what, i)

    eq = oracle.prepare_alias(g.row_ptr, np.full(g.ne, 3.0, dtype=np.float32), lib=lib)
    same(oracle.walk(g.row_ptr, g.col, oracle.DEEPWALK_WEIGHTED, src, L, seed=3, alias=eq, lib=lib),
         "alias with equal weights")
    w3 = np.full(g.ne, 3.0, dtype=np.float32)
    same(oracle.walk(g.row_ptr, g.col, oracle.DEEPWALK_WEIGHTED, src, L, seed=3, sampler=oracle.SAMPLER_ITS,
                     its=oracle.prepare_its(g.row_ptr, w3, lib=lib), lib=lib), "its with equal weights")
    same(oracle.walk(g.row_ptr, g.col, oracle.DEEPWALK_WEIGHTED, src, L, seed=3, sampler=oracle.SAMPLER_REJ,
                     pmax=oracle.prepare_rej(g.row_ptr, w3, lib=lib), weights=w3, lib=lib), "rej with equal weights")
    same(oracle.walk(g.row_ptr, g.col, oracle.DEEPWALK_WEIGHTED, src, L, seed=3, sampler=oracle.SAMPLER_OREJ,
                     weights=w3, max_weight=3.0, lib=lib), "o-rej with equal weights at the bound")
    same(oracle.walk(g.row_ptr, g.col, oracle.METAPATH, src, L, seed=3, labels=np.zeros(g.ne, np.uint8),
                     schema=[0], lib=lib), "metapath on one label")
    same(oracle.walk(g.row_ptr, g.col, oracle.NODE2VEC, src, L, seed=3, n2v_p=1.0, n2v_q=1.0, lib=lib),
         "node2vec p=q=1")
    same(oracle.walk(g.row_ptr, g.col, oracle.PPR, src, L, seed=3, ppr_stop=0.0, lib=lib), "ppr stop 0")


def pin_invariants(lib=None):
    """Every hop is an edge, lengths are bounded, MetaPath hops carry the
    schema's label, and walks end early only where the rules say so."""
    g = small_rmat()
    al = oracle.prepare_alias(g.row_ptr, g.weights, lib=lib)
    src = synth.vertex_sources(g.nv)
    schema = np.array([1, 3, 0, 4, 2], dtype=np.uint8)
    L = 30
    adj = [set(nbrs(g, v)) for v in range(g.nv)]
    lab = {}
    for v in range(g.nv):
        for j in range(int(g.row_ptr[v]), int(g.row_ptr[v + 1])):
            lab[(v, int(g.col[j]))] = int(g.labels[j])
    for algo, kw in [(oracle.DEEPWALK, {}), (oracle.DEEPWALK_WEIGHTED, {"alias": al}),
                     (oracle.PPR, {"ppr_stop": 0.2}), (oracle.NODE2VEC, {"n2v_p": 0.5, "n2v_q": 2.0}),
                     (oracle.METAPATH, {"labels": g.labels, "schema": schema})]:
        res = oracle.walk(g.row_ptr, g.col, algo, src, L, seed=21, lib=lib, **kw)
        assert res.status == 0
        assert res.stats["moves"] == int((res.lengths - 1).sum())
        for i in range(g.nv):
            ln = int(res.lengths[i])
            assert 1 <= ln <= L + 1
            path = res.paths[i, :ln]
            assert path[0] == src[i]
            for s in range(ln - 1):
                a, b = int(path[s]), int(path[s + 1])
                assert b in adj[a], (algo, i, s)
                if algo == oracle.METAPATH:
                    assert lab[(a, b)] == schema[s % len(schema)]
            if ln < L + 1 and algo in (oracle.DEEPWALK, oracle.DEEPWALK_WEIGHTED, oracle.NODE2VEC):
                assert not adj[int(path[-1])], "early stop only at a dead end"
            if ln < L + 1 and algo == oracle.METAPATH:
                v = int(path[-1])
                h = schema[(ln - 1) % len(schema)]
                assert all(lab[(v, c)] != h for c in adj[v]), "early stop only without a matching label"


def pin_sharding(lib=None):
    """A walk depends only on (seed, walk index): splitting the batch with
    walk_offset reproduces the whole batch (Node2Vec, weighted Node2Vec and
    weighted DeepWalk under ITS, REJ and O-REJ)."""
    g = small_rmat()
    src = synth.vertex_sources(g.nv)
    tabs = {"weights": g.weights, "its": oracle.prepare_its(g.row_ptr, g.weights, lib=lib),
            "pmax": oracle.prepare_rej(g.row_ptr, g.weights, lib=lib)}
    cases = [(oracle.NODE2VEC, {"n2v_p": 0.5, "n2v_q": 2.0}),
             (oracle.NODE2VEC_WEIGHTED, dict(tabs, n2v_p=2.0, n2v_q=0.5)),
             (oracle.DEEPWALK_WEIGHTED, dict(tabs, sampler=oracle.SAMPLER_ITS)),
             (oracle.DEEPWALK_WEIGHTED, dict(tabs, sampler=oracle.SAMPLER_REJ)),
             (oracle.DEEPWALK_WEIGHTED, dict(tabs, sampler=oracle.SAMPLER_OREJ, max_weight=100.0))]
    for algo, kw in cases:
        full = oracle.walk(g.row_ptr, g.col, algo, src, 12, seed=9, lib=lib, **kw)
        a = oracle.walk(g.row_ptr, g.col, algo, src[:300], 12, seed=9, lib=lib, **kw)
        b = oracle.walk(g.row_ptr, g.col, algo, src[300:], 12, seed=9, walk_offset=300, lib=lib, **kw)
        assert full.status == a.status == b.status == 0
        assert np.array_equal(np.concatenate([a.lengths, b.lengths]), full.lengths), algo
        for i in range(g.nv):
            part = a if i < 300 else b
            j = i if i < 300 else i - 300
            ln = full.lengths[i]
            assert np.array_equal(part.paths[j, :ln], full.paths[i, :ln]), (algo, i)


# ------------------------------------------- ITS, REJ and O-REJ (Section 2.3)

def _wq(w):
    """Integer weights by numpy: round-half-even(w * 2^16), clamped."""
    return np.minimum(np.rint(np.asarray(w, dtype=np.float32).astype(np.float64) * 65536.0), TWO32 - 1).astype(
        np.int64)


def _r64(B):
    return int(B[0]) | (int(B[1]) << 32)


# ------------------------------------------------------------- sector model
# The oracle's statistics count, per move, the distinct 32-byte sectors the
# device layout reads (4-byte row offsets and vertex ids, 16-byte packed alias
# records, 8-byte ITS prefix sums, 4-byte REJ bounds and weights, 1-byte
# labels), and the bytes of path output.  The counts below are worked out by
# hand on graphs built so that the count does not depend on which neighbour a
# draw picks; each comment gives the byte ranges.

def _cycle(nv=10):
    return synth.from_edges(nv, [(v, (v + 1) % nv) for v in range(nv)], symmetric=False)


def pin_sector_model(lib=None):
    """stats.sectors and stats.out_bytes against hand counts (the per-step
    access chains of Section 2.3's samplers on the device layout)."""
    g = _cycle()
    src = np.arange(10, dtype=np.int32)
    ones = np.ones(g.ne, dtype=np.float32)

    def run(algo, L, **kw):
        res = oracle.walk(g.row_ptr, g.col, algo, src, L, seed=11, lib=lib, **kw)
        assert res.status == 0
        return res.stats

    # Cycle v -> v+1: every move reads the row pair of v (bytes 4v..4v+7: one
    # sector, two for v = 7, whose pair straddles byte 32) and one more
    # sector per array the sampler reads (a row of one edge).
    st = run(oracle.DEEPWALK, 1)
    assert (st["moves"], st["sectors"], st["out_bytes"]) == (10, 21, 80), st
    # Three moves from each vertex: 30 moves, and vertex 7 starts a move of
    # the walks from 5, 6 and 7.  Paths of 4 vertices: 10 * 16 bytes.
    st = run(oracle.DEEPWALK, 3)
    assert (st["moves"], st["sectors"], st["out_bytes"]) == (30, 63, 160), st
    st = run(oracle.PPR, 3, ppr_stop=0.0, endpoints_only=True)
    assert (st["moves"], st["sectors"], st["out_bytes"]) == (30, 63, 40), st
    # ALIAS: the row pair and one packed record (its destination inside).
    al = oracle.prepare_alias(g.row_ptr, ones, lib=lib)
    st = run(oracle.DEEPWALK_WEIGHTED, 1, alias=al)
    assert (st["moves"], st["sectors"]) == (10, 21), st
    # ITS on a one-edge row: the row pair, P'_{d-1}, the picked id.
    st = run(oracle.DEEPWALK_WEIGHTED, 1, sampler=oracle.SAMPLER_ITS, its=oracle.prepare_its(g.row_ptr, ones, lib=lib))
    assert (st["moves"], st["sectors"]) == (10, 31), st
    # REJ: the row pair, p*_v, then the dart's weight and id (a dart on the
    # row's largest weight always hits).
    st = run(oracle.DEEPWALK_WEIGHTED, 1, sampler=oracle.SAMPLER_REJ, weights=ones,
             pmax=oracle.prepare_rej(g.row_ptr, ones, lib=lib))
    assert (st["moves"], st["attempts"], st["sectors"]) == (10, 10, 41), st
    # O-REJ: as REJ without p*_v (the caller's bound).
    st = run(oracle.DEEPWALK_WEIGHTED, 1, sampler=oracle.SAMPLER_OREJ, weights=ones, max_weight=1.0)
    assert (st["moves"], st["attempts"], st["sectors"]) == (10, 10, 31), st

    # ITS binary search: 0 -> 1..16, all weight on the edge at index 12.
    # P' = 0 (indices 0..11), then W.  Probes: P'_15 (byte 120), then the
    # lower-bound search over [0, 15): 7 (byte 56), 11 (88), 13 (104),
    # 12 (96): sectors 1, 2, 3.  The id at index 12 is at byte 48 (sector 1)
    # and the row pair of 0 in sector 0: 5 sectors a move.
    gs = synth.from_edges(17, [(0, c) for c in range(1, 17)], symmetric=False)
    w = np.zeros(16, dtype=np.float32)
    w[12] = 1.0
    res = oracle.walk(gs.row_ptr, gs.col, oracle.DEEPWALK_WEIGHTED, [0], 1, seed=5, walks_per_source=6,
                      sampler=oracle.SAMPLER_ITS, its=oracle.prepare_its(gs.row_ptr, w, lib=lib), lib=lib)
    assert res.status == 0 and np.all(res.paths[:, 1] == 13)
    assert (res.stats["moves"], res.stats["sectors"]) == (6, 30), res.stats

    # MetaPath: vertex 0 has 31 edges, so vertex 1's two edges sit at
    # indices 31 and 32: its labels span bytes 31..32 (sectors 0 and 1), its
    # ids bytes 124..131 (one sector either way), its row pair bytes 4..11.
    # Vertex 0: labels bytes 0..30, one sector.
    gm = synth.from_edges(33, [(0, c) for c in range(2, 33)] + [(1, 2), (1, 3)], symmetric=False)
    lab = np.zeros(gm.ne, dtype=np.uint8)
    for s0, per in ((1, 4), (0, 3)):
        res = oracle.walk(gm.row_ptr, gm.col, oracle.METAPATH, [s0], 1, seed=5, walks_per_source=4, labels=lab,
                          schema=[0], lib=lib)
        assert res.status == 0
        assert (res.stats["moves"], res.stats["sectors"]) == (4, 4 * per), (s0, res.stats)

    # Node2Vec IsNeighbor: N(0) = {1, 3, 4, 5, 6, 8..18} (16 ids, bytes
    # 0..63), vertices 1, 3, 4, 5, 6 each lead only to 2, and 2 is not in
    # N(0).  First move from 0: row pair (sector 0) and one id: 2 sectors.
    # Second move from v in {1, 3, 4, 5, 6} (vertices 8..18 are dead ends):
    # every dart draws 2 (ids at indices 16..21, sector 2); IsNeighbor(2, 0)
    # reads 0's row pair (sector 0, as v's) and probes indices 8, 4, 2, 1, 0
    # (sectors 1 and 0): 4 sectors, however many darts the step throws.
    n0 = [1, 3, 4, 5, 6] + list(range(8, 19))
    gn = synth.from_edges(19, [(0, c) for c in n0] + [(v, 2) for v in (1, 3, 4, 5, 6)] + [(2, 0)], symmetric=False)
    n = 2000
    res = oracle.walk(gn.row_ptr, gn.col, oracle.NODE2VEC, [0], 2, seed=9, walks_per_source=n, n2v_p=0.5,
                      n2v_q=2.0, lib=lib)
    assert res.status == 0
    second = res.stats["moves"] - n
    assert 0 < second < n
    assert res.stats["attempts"] > res.stats["moves"]  # some darts were rejected
    assert res.stats["sectors"] == 2 * n + 4 * second, res.stats


def pin_return_only_count(lib=None):
    """stats.return_only (unweighted Node2Vec darts after the first move whose
    word is at or past both non-return thresholds): zero where no such word
    exists (p = q = 1, or a non-return class with weight p*, or one move per
    walk), else a fraction 1 - T_hi / 2^32 of the darts after the first move,
    T_hi = floor(max(w_nb, w_far) / p* * 2^32)."""
    g = small_rmat()
    src = synth.vertex_sources(g.nv)

    def st(L, pp, qq):
        res = oracle.walk(g.row_ptr, g.col, oracle.NODE2VEC, src, L, seed=7, n2v_p=pp, n2v_q=qq, lib=lib)
        assert res.status == 0
        return res.stats

    for pp, qq in ((1.0, 1.0), (2.0, 0.5), (1.0, 0.5)):
        assert st(30, pp, qq)["return_only"] == 0, (pp, qq)
    assert st(1, 0.5, 2.0)["return_only"] == 0
    for pp, qq, frac in ((0.5, 2.0, 0.5), (0.25, 4.0, 0.75)):
        first = st(1, pp, qq)["attempts"]  # the first move takes one dart (Weight = MaxWeight)
        s = st(30, pp, qq)
        later = s["attempts"] - first
        assert later > 20000
        got = s["return_only"] / later
        assert abs(got - frac) < 6 * np.sqrt(frac * (1 - frac) / later), (pp, qq, got, frac)


def pin_rej_threshold(lib=None):
    """T = rej_threshold(W, p*) is the number of 32-bit words y with
    (y + 1) / 2^32 <= W / p*: word T - 1 passes and word T fails."""
    cases = [(1, 3), (2, 3), (5, 7), (65536, 6553600), (6553599, 6553600), (123457, 999983), (TWO32 - 2, TWO32 - 1),
             (1, TWO32 - 1), (7, 7), (9, 7), (0, 5), (65536 * 3, 65536 * 4)]
    for W, ps in cases:
        T = oracle.rej_threshold(W, ps, lib=lib)
        if W >= ps:
            assert T == TWO32, (W, ps)
            continue
        assert 0 <= T < TWO32
        if T > 0:
            assert T * ps <= W * TWO32, (W, ps, T)          # y = T - 1 passes
        assert (T + 1) * ps > W * TWO32, (W, ps, T)          # y = T fails


def pin_its_first_move(lib=None):
    """Every ITS walk's first move equals numpy's searchsorted over the
    cumulative integer weights at x = floor(r64 * S / 2^64)."""
    g = small_rmat()
    cdf = oracle.prepare_its(g.row_ptr, g.weights, lib=lib)
    src = synth.vertex_sources(g.nv)
    seed = 0x1234567890ABCDEF
    res = oracle.walk(g.row_ptr, g.col, oracle.DEEPWALK_WEIGHTED, src, 1, seed, sampler=oracle.SAMPLER_ITS, its=cdf,
                      lib=lib)
    assert res.status == 0
    Wq = _wq(g.weights)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i, v in enumerate(src):
        lo, hi = int(g.row_ptr[v]), int(g.row_ptr[v + 1])
        if hi == lo:
            assert res.lengths[i] == 1
            continue
        P = np.cumsum(Wq[lo:hi])
        S = int(P[-1])
        B = oracle.philox4x32_10([i, 0, 0, 0], key)
        x = (_r64(B) * S) >> 64
        j = int(np.searchsorted(P, x, side="right"))
        assert res.lengths[i] == 2 and res.paths[i, 1] == g.col[lo + j], (i, v)


def _darts(g, Wq, v, key, walk, step, pstar):
    """REJ dart sequence of one step with the acceptance test written as
    (y + 1) * p* <= W_x * 2^32; returns (edge slot, trials)."""
    lo, hi = int(g.row_ptr[v]), int(g.row_ptr[v + 1])
    d = hi - lo
    for a in range(65536):
        B = oracle.philox4x32_10([walk, step, a, 0], key)
        x = (_r64(B) * d) >> 64
        if (int(B[2]) + 1) * pstar <= int(Wq[lo + x]) * TWO32:
            return lo + x, a + 1
    raise AssertionError("trial cap")


def pin_rej_first_move(lib=None):
    """Every REJ and O-REJ walk's first move, and the trials it took, from the
    dart sequence recomputed in Python (p* the row maximum by numpy for REJ,
    the quantised bound for O-REJ)."""
    g = small_rmat()
    pm = oracle.prepare_rej(g.row_ptr, g.weights, lib=lib)
    src = synth.vertex_sources(g.nv)[:400]
    seed = 77
    key = [seed, 0]
    Wq = _wq(g.weights)
    for sampler, bound in ((oracle.SAMPLER_REJ, None), (oracle.SAMPLER_OREJ, 130.5)):
        res = oracle.walk(g.row_ptr, g.col, oracle.DEEPWALK_WEIGHTED, src, 1, seed, sampler=sampler, weights=g.weights,
                          pmax=pm if sampler == oracle.SAMPLER_REJ else None, max_weight=bound or 0.0, lib=lib)
        assert res.status == 0
        trials = 0
        for i, v in enumerate(src):
            lo, hi = int(g.row_ptr[v]), int(g.row_ptr[v + 1])
            if hi == lo:
                assert res.lengths[i] == 1
                continue
            ps = int(Wq[lo:hi].max()) if bound is None else int(np.rint(bound * 65536))
            e, t = _darts(g, Wq, int(v), key, i, 0, ps)
            trials += t
            assert res.lengths[i] == 2 and res.paths[i, 1] == g.col[e], (sampler, i)
        assert res.stats["attempts"] == trials, sampler


def _sweep_laws(g, lib):
    cdf = oracle.prepare_its(g.row_ptr, g.weights, lib=lib)
    pm = oracle.prepare_rej(g.row_ptr, g.weights, lib=lib)
    return [(oracle.SAMPLER_ITS, {"its": cdf}), (oracle.SAMPLER_REJ, {"pmax": pm, "weights": g.weights}),
            (oracle.SAMPLER_OREJ, {"weights": g.weights, "max_weight": 12.0})]


def pin_law_samplers(lib=None):
    """Three-move path laws of ITS, REJ and O-REJ equal the weighted law
    w_e / sum(w) of Section 2.2 (chi-square on the directed graph, whose
    weights are exact in fixed point)."""
    g = dir_graph()

    def law(path):
        v = path[-1]
        nb = nbrs(g, v)
        ws = [DIR_WEIGHTS[(v, c)] for c in nb]
        return {c: w / sum(ws) for c, w in zip(nb, ws)}

    want = enumerate_paths(0, 3, law)
    for sampler, kw in _sweep_laws(g, lib):
        res = oracle.walk(g.row_ptr, g.col, oracle.DEEPWALK_WEIGHTED, [0], 3, seed=31 + sampler, walks_per_source=N_LAW,
                          sampler=sampler, lib=lib, **kw)
        assert res.status == 0, sampler
        p = chi2_pvalue(path_counts(res), want, N_LAW)
        assert p > 1e-3, (sampler, p)


def pin_rej_trials_closed_form(lib=None):
    """On a circulant graph whose every row holds the weights {1, 3, 4}, the
    mean trials per move are d * p* / sum(p) (Section 2.3): 3 * 4 / 8 = 1.5 for
    REJ (p* = 4) and 3 * 8 / 8 = 3 for O-REJ with the bound 8."""
    n = 64
    edges = [(v, (v + k) % n) for v in range(n) for k in (1, 2, 3)]
    g = synth.from_edges(n, edges, symmetric=False)
    wmap = {(v, (v + k) % n): float(w) for v in range(n) for k, w in ((1, 1), (2, 3), (3, 4))}
    g.weights = np.array([wmap[(v, int(c))] for v in range(n) for c in g.col[g.row_ptr[v]:g.row_ptr[v + 1]]],
                         dtype=np.float32)
    pm = oracle.prepare_rej(g.row_ptr, g.weights, lib=lib)
    L, walks = 20, 4000
    for sampler, kw, e in ((oracle.SAMPLER_REJ, {"pmax": pm}, 1.5), (oracle.SAMPLER_OREJ, {"max_weight": 8.0}, 3.0)):
        res = oracle.walk(g.row_ptr, g.col, oracle.DEEPWALK_WEIGHTED, np.arange(n), L, seed=5, walks_per_source=walks // n,
                          sampler=sampler, weights=g.weights, lib=lib, **kw)
        assert res.status == 0
        moves = res.stats["moves"]
        assert moves == walks // n * n * L
        q = 1.0 / e
        var = (1 - q) / q ** 2
        got = res.stats["attempts"] / moves
        assert abs(got - e) < 6 * np.sqrt(var / moves), (sampler, got, e)


def pin_zero_weights(lib=None):
    """Zero-weight edges are never taken; a row of only zero weights is a dead
    end for ALIAS, ITS and REJ, and exhausts O-REJ's trial cap."""
    edges = [(0, 1), (0, 2), (0, 3), (0, 4), (1, 0), (1, 2), (2, 1), (3, 0), (4, 0)]
    g = synth.from_edges(5, edges, symmetric=False)
    wmap = {(0, 1): 0.0, (0, 2): 2.0, (0, 3): 0.0, (0, 4): 5.0, (1, 0): 1.0, (1, 2): 1.0, (2, 1): 1.0,
            (3, 0): 1.0, (4, 0): 0.0}
    w = np.array([wmap[(v, int(c))] for v in range(5) for c in g.col[g.row_ptr[v]:g.row_ptr[v + 1]]], np.float32)
    al = oracle.prepare_alias(g.row_ptr, w, lib=lib)
    cdf = oracle.prepare_its(g.row_ptr, w, lib=lib)
    pm = oracle.prepare_rej(g.row_ptr, w, lib=lib)
    assert list(pm) == [5 * 65536, 65536, 65536, 65536, 0]
    for sampler, kw in ((oracle.SAMPLER_DEFAULT, {"alias": al}), (oracle.SAMPLER_ITS, {"its": cdf}),
                        (oracle.SAMPLER_REJ, {"pmax": pm, "weights": w})):
        res = oracle.walk(g.row_ptr, g.col, oracle.DEEPWALK_WEIGHTED, [0], 5, seed=4, walks_per_source=2000,
                          sampler=sampler, lib=lib, **kw)
        assert res.status == 0, sampler
        firsts = Counter(int(x) for x in res.paths[:, 1])
        assert set(firsts) == {2, 4}, (sampler, firsts)
        for row, ln in zip(res.paths, res.lengths):
            if 4 in row[:ln]:
                assert row[ln - 1] == 4 and ln == list(row[:ln]).index(4) + 1, "a zero row ends the walk"
            else:
                assert ln == 6
    res = oracle.walk(g.row_ptr, g.col, oracle.DEEPWALK_WEIGHTED, [4], 3, seed=4, sampler=oracle.SAMPLER_OREJ,
                      weights=w, max_weight=5.0, lib=lib)
    assert res.status == oracle.ERR_REJECT_CAP


# ------------------------------------------------ weighted Node2Vec (Section 2.2)

def node2vec_weighted_step_law(g, path, p_ret, q_io, bound):
    """Eq. 1 times the edge weight, in the fixed point of its O-REJ dart: a
    candidate c passes the class word with T_class(c) / 2^32 and the weight
    word with floor(W_c 2^32 / P) / 2^32; P = bound(v) (p*_v or the caller's)."""
    v = path[-1]
    nb = nbrs(g, v)
    if not nb:
        return {}
    P = bound(v)
    wt = {c: min(TWO32, (int(round(DIR_WEIGHTS[(v, c)] * 65536)) << 32) // P) for c in nb}
    if len(path) == 1:
        t = {c: TWO32 for c in nb}
    else:
        u = path[-2]
        w_ret, w_nb, w_far = 1.0 / p_ret, 1.0, 1.0 / q_io
        pstar = max(w_ret, w_nb, w_far)
        T = {k: (Fraction(x / pstar) * TWO32).__floor__() for k, x in (("r", w_ret), ("n", w_nb), ("f", w_far))}
        nu = set(nbrs(g, u))
        t = {c: T["r"] if c == u else (T["n"] if c in nu else T["f"]) for c in nb}
    tot = sum(t[c] * wt[c] for c in nb)
    return {c: t[c] * wt[c] / tot for c in nb}


def pin_law_node2vec_weighted(lib=None):
    """Three-move path laws of weighted Node2Vec with the REJ bound p*_v and
    with a caller's bound, by chi-square against the exact product law."""
    g = dir_graph()
    pm = oracle.prepare_rej(g.row_ptr, g.weights, lib=lib)
    for (pp, qq, seed, mw) in [(0.5, 2.0, 23, 0.0), (2.0, 0.5, 24, 12.0)]:
        res = oracle.walk(g.row_ptr, g.col, oracle.NODE2VEC_WEIGHTED, [0], 3, seed=seed, walks_per_source=N_LAW,
                          n2v_p=pp, n2v_q=qq, weights=g.weights, pmax=pm, max_weight=mw, lib=lib)
        assert res.status == 0
        bound = (lambda v: int(pm[v])) if mw == 0.0 else (lambda v: int(round(mw * 65536)))
        law = enumerate_paths(0, 3, lambda path: node2vec_weighted_step_law(g, path, pp, qq, bound))
        p = chi2_pvalue(path_counts(res), law, N_LAW)
        assert p > 1e-3, (pp, qq, mw, p)


def pin_node2vec_weighted_first_move(lib=None):
    """The first move of every weighted Node2Vec walk, and its trials, from the
    dart sequence recomputed in Python: x from words 0-1, the weight word 3
    tested as (z + 1) * P <= W_x * 2^32 (the class passes at the source)."""
    g = small_rmat()
    pm = oracle.prepare_rej(g.row_ptr, g.weights, lib=lib)
    src = synth.vertex_sources(g.nv)[:300]
    seed = 5
    Wq = _wq(g.weights)
    res = oracle.walk(g.row_ptr, g.col, oracle.NODE2VEC_WEIGHTED, src, 1, seed, n2v_p=0.5, n2v_q=2.0,
                      weights=g.weights, pmax=pm, lib=lib)
    assert res.status == 0
    trials = 0
    for i, v in enumerate(src):
        lo, hi = int(g.row_ptr[v]), int(g.row_ptr[v + 1])
        if hi == lo:
            continue
        d = hi - lo
        ps = int(Wq[lo:hi].max())
        for a in range(65536):
            B = oracle.philox4x32_10([i, 0, a, 0], [seed, 0])
            x = (_r64(B) * d) >> 64
            if (int(B[3]) + 1) * ps <= int(Wq[lo + x]) * TWO32:
                break
        trials += a + 1
        assert res.paths[i, 1] == g.col[lo + x], i
    assert res.stats["attempts"] == trials


def pin_node2vec_weighted_reductions(lib=None):
    """Every weight equal to the bound: unweighted Node2Vec's walks, bit for bit
    (the weight word always passes); with p = q = 1 and equal weights, the
    trials per move are d P / sum(W) = 1."""
    g = small_rmat()
    src = synth.vertex_sources(g.nv)
    w3 = np.full(g.ne, 3.0, dtype=np.float32)
    base = oracle.walk(g.row_ptr, g.col, oracle.NODE2VEC, src, 15, seed=8, n2v_p=0.5, n2v_q=2.0, lib=lib)
    for kw in ({"max_weight": 3.0}, {"pmax": oracle.prepare_rej(g.row_ptr, w3, lib=lib)}):
        res = oracle.walk(g.row_ptr, g.col, oracle.NODE2VEC_WEIGHTED, src, 15, seed=8, n2v_p=0.5, n2v_q=2.0,
                          weights=w3, lib=lib, **kw)
        assert res.status == 0 and np.array_equal(res.lengths, base.lengths)
        mask = np.arange(16)[None, :] < base.lengths[:, None]
        assert np.array_equal(res.paths[mask], base.paths[mask]), kw
        assert res.stats["attempts"] == base.stats["attempts"]


# ---------------------------------------------- user-defined walks (Section 4.3)

def pin_custom_walk_reductions(lib=None):
    """User functions that restate a built-in walk give its walks bit for bit:
    NAIVE with no Update (DeepWalk), an Update that stops after 7 moves
    (DeepWalk truncated), O-REJ with Eq. 1's weights in fixed point 4 / 2 / 1
    over MaxWeight 4 (Node2Vec a = 0.5, b = 2), O-REJ with the integer edge
    weights over the quantised bound (weighted DeepWalk under O-REJ)."""
    g = small_rmat()
    src = synth.vertex_sources(g.nv)
    L = 12

    def same(res, base, what, L=L):
        assert res.status == 0 and base.status == 0, what
        assert np.array_equal(res.lengths, base.lengths), what
        mask = np.arange(L + 1)[None, :] < base.lengths[:, None]
        assert np.array_equal(res.paths[:, :L + 1][mask], base.paths[mask]), what

    dw = oracle.walk(g.row_ptr, g.col, oracle.DEEPWALK, src, L, seed=4, lib=lib)
    same(oracle.walk_custom(g.row_ptr, g.col, src, L, 4, sampler=oracle.NAIVE_SAMPLER, lib=lib), dw, "naive")
    dw7 = oracle.walk(g.row_ptr, g.col, oracle.DEEPWALK, src, 7, seed=4, lib=lib)
    res = oracle.walk_custom(g.row_ptr, g.col, src, L, 4, sampler=oracle.NAIVE_SAMPLER,
                             update=lambda w, ln, cur, prev, dst, e: ln == 7, lib=lib)
    same(res, dw7, "update at 7", L=7)
    adj = [set(nbrs(g, v)) for v in range(g.nv)]

    def n2v_weight(w, ln, cur, prev, dst, e):
        if ln == 0:
            return 4
        return 4 if dst == prev else (2 if dst in adj[prev] else 1)

    n2v = oracle.walk(g.row_ptr, g.col, oracle.NODE2VEC, src, L, seed=6, n2v_p=0.5, n2v_q=2.0, lib=lib)
    same(oracle.walk_custom(g.row_ptr, g.col, src, L, 6, sampler=oracle.OREJ_SAMPLER, weight=n2v_weight,
                            max_weight=4, lib=lib), n2v, "node2vec")
    Wq = _wq(g.weights)
    orej = oracle.walk(g.row_ptr, g.col, oracle.DEEPWALK_WEIGHTED, src, L, seed=8, sampler=oracle.SAMPLER_OREJ,
                       weights=g.weights, max_weight=100.0, lib=lib)
    same(oracle.walk_custom(g.row_ptr, g.col, src, L, 8, sampler=oracle.OREJ_SAMPLER,
                            weight=lambda w, ln, cur, prev, dst, e: int(Wq[e]), max_weight=100 * 65536, lib=lib),
         orej, "weighted o-rej")


def pin_custom_walk_update(lib=None):
    """Update sees the moved query and ends the walk exactly at the first
    vertex it accepts; the Weight law of O-REJ by chi-square (a weight of
    both endpoints, 1 + 3 ((cur + 2 dst) mod 3) over MaxWeight 7, on the
    directed graph)."""
    g = small_rmat()
    src = synth.vertex_sources(g.nv)
    seen = []

    def upd(w, ln, cur, prev, dst, e):
        seen.append((ln, cur, dst))
        return cur % 5 == 0

    res = oracle.walk_custom(g.row_ptr, g.col, src, 30, 2, sampler=oracle.NAIVE_SAMPLER, update=upd, lib=lib)
    assert res.status == 0 and all(cur == dst for _, cur, dst in seen)
    for row, ln in zip(res.paths, res.lengths):
        path = [int(x) for x in row[:ln]]
        stops = [k for k in range(1, len(path)) if path[k] % 5 == 0]
        if stops:
            assert len(path) - 1 == stops[0]
        else:
            assert len(path) == 31 or not nbrs(g, path[-1])
    gd = dir_graph()
    res = oracle.walk_custom(gd.row_ptr, gd.col, [0], 2, 3, sampler=oracle.OREJ_SAMPLER,
                             weight=lambda w, ln, cur, prev, dst, e: 1 + 3 * ((cur + 2 * dst) % 3), max_weight=7,
                             walks_per_source=N_LAW, lib=lib)
    assert res.status == 0

    def law(path):
        v = path[-1]
        nb = nbrs(gd, v)
        t = {c: 1 + 3 * ((v + 2 * c) % 3) for c in nb}
        return {c: t[c] / sum(t.values()) for c in nb}

    p = chi2_pvalue(path_counts(res), enumerate_paths(0, 2, law), N_LAW)
    assert p > 1e-3, p


ALL_PINS = [pin_philox_kat, pin_fixed_point, pin_sector_model, pin_return_only_count, pin_alias_law, pin_law_deepwalk, pin_law_alias, pin_law_node2vec,
            pin_law_metapath, pin_ppr, pin_rejection_trials, pin_reductions, pin_invariants, pin_sharding, pin_rej_threshold, pin_its_first_move,
            pin_rej_first_move, pin_law_samplers, pin_rej_trials_closed_form, pin_zero_weights,
            pin_law_node2vec_weighted, pin_node2vec_weighted_first_move, pin_node2vec_weighted_reductions,
            pin_custom_walk_reductions, pin_custom_walk_update]
