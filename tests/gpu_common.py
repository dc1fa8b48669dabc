"""Helpers of the GPU parity tests: graphs, oracle runs, element-wise comparison."""
from __future__ import annotations

import functools

import numpy as np

import oracle
import synth

ORACLE_ALGO = {0: oracle.DEEPWALK, 1: oracle.DEEPWALK_WEIGHTED, 2: oracle.PPR, 3: oracle.NODE2VEC, 4: oracle.METAPATH}


@functools.lru_cache(maxsize=None)
def rmat_graph(scale: int, seed: int = 42, symmetric: bool = True, nlabels: int = 5):
    g = synth.rmat(scale, seed=seed, symmetric=symmetric)
    g.weights = synth.edge_weights(g, seed=seed)
    g.labels = synth.edge_labels(g, seed=seed, nlabels=nlabels)
    return g


@functools.lru_cache(maxsize=None)
def oracle_alias(scale: int, seed: int = 42, symmetric: bool = True):
    g = rmat_graph(scale, seed, symmetric)
    return oracle.prepare_alias(g.row_ptr, g.weights)


def oracle_walk(g, algo, sources, max_len, seed, alias=None, **kw):
    res = oracle.walk(g.row_ptr, g.col, ORACLE_ALGO[algo], sources, max_len, seed, alias=alias,
                      labels=g.labels, **kw)
    assert res.status == 0, res.status
    return res


def assert_paths_equal(got_paths, got_lengths, want, endpoints=False):
    gp = np.asarray(got_paths)
    gl = np.asarray(got_lengths)
    assert gl.shape == want.lengths.shape
    bad = np.nonzero(gl != want.lengths)[0]
    assert bad.size == 0, f"{bad.size} lengths differ, first walk {bad[0]}: {gl[bad[0]]} vs {want.lengths[bad[0]]}"
    if endpoints:
        bad = np.nonzero(gp != want.paths)[0]
        assert bad.size == 0, f"{bad.size} endpoints differ, first walk {bad[0]}"
        return
    L1 = want.paths.shape[1]
    mask = np.arange(L1)[None, :] < want.lengths[:, None]
    diff = (gp != want.paths) & mask
    rows = np.nonzero(diff.any(axis=1))[0]
    assert rows.size == 0, (f"{rows.size} paths differ; first walk {rows[0]}: got {gp[rows[0], :gl[rows[0]]]} "
                            f"want {want.paths[rows[0], :want.lengths[rows[0]]]}")
