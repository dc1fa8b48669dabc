"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

Holds no arithmetic of the walk method: R-MAT graphs as sorted, de-duplicated
CSR, per-edge fp32 weights and uint8 labels keyed on the unordered endpoint
pair, uniform walk sources and MetaPath schemas.  All of it comes from
``synth.c`` (compiled on first use with gcc) through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB_PATH = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

# R-MAT quadrant probabilities and edge factor of every workload here.
RMAT_A, RMAT_B, RMAT_C = 0.57, 0.19, 0.19
EDGE_FACTOR = 16
GRAPH_SEED = 42


def build(force: bool = False) -> str:
    """Compile libsynth.so next to its source (gcc, pthreads)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-std=gnu11", "-Wall", "-shared", "-fPIC", "-pthread",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i64p = ctypes.POINTER(ctypes.c_int64)
            lib.syn_rmat_build.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_void_p, i64p, ctypes.POINTER(ctypes.c_void_p)]
            lib.syn_rmat_build.restype = ctypes.c_int
            lib.syn_free.argtypes = [ctypes.c_void_p]
            lib.syn_edge_weights.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                             ctypes.c_float, ctypes.c_float, ctypes.c_void_p, ctypes.c_int]
            lib.syn_edge_labels.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                            ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
            lib.syn_sources.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p]
            lib.syn_schema.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p]
            lib.syn_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64]
            lib.syn_draw.restype = ctypes.c_uint64
            _lib = lib
    return _lib


@dataclass
class Graph:
    """A CSR graph: row_ptr int64[nv+1], col int32[ne] (rows sorted, no duplicates)."""

    row_ptr: np.ndarray
    col: np.ndarray
    weights: Optional[np.ndarray] = None  # fp32[ne]
    labels: Optional[np.ndarray] = None   # uint8[ne]
    name: str = ""

    @property
    def nv(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def ne(self) -> int:
        return int(self.col.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)


def rmat(scale: int, edge_factor: int = EDGE_FACTOR, a: float = RMAT_A, b: float = RMAT_B,
         c: float = RMAT_C, seed: int = GRAPH_SEED, symmetric: bool = True, nthreads: int = 0) -> Graph:
    """R-MAT graph with 2**scale vertices and edge_factor*2**scale generated edges."""
    lib = _load()
    nv = 1 << scale
    row_ptr = np.empty(nv + 1, dtype=np.int64)
    ne = ctypes.c_int64(0)
    colp = ctypes.c_void_p(0)
    rc = lib.syn_rmat_build(scale, edge_factor, a, b, c, seed, int(symmetric), nthreads,
                            row_ptr.ctypes.data, ctypes.byref(ne), ctypes.byref(colp))
    if rc != 0:
        raise RuntimeError(f"syn_rmat_build failed with {rc}")
    n = ne.value
    col = np.empty(n, dtype=np.int32)
    if n:
        ctypes.memmove(col.ctypes.data, colp.value, n * 4)
    lib.syn_free(colp)
    kind = "sym" if symmetric else "dir"
    return Graph(row_ptr=row_ptr, col=col, name=f"rmat-s{scale}-ef{edge_factor}-{kind}")


def edge_weights(g: Graph, seed: int = GRAPH_SEED, lo: float = 1.0, hi: float = 100.0,
                 nthreads: int = 0) -> np.ndarray:
    """fp32 weight per edge, uniform in [lo, hi), equal on both directions of a pair."""
    lib = _load()
    w = np.empty(g.ne, dtype=np.float32)
    rc = lib.syn_edge_weights(g.nv, g.row_ptr.ctypes.data, g.col.ctypes.data, seed, lo, hi,
                              w.ctypes.data, nthreads)
    if rc != 0:
        raise ValueError("bad weight range")
    return w


def edge_labels(g: Graph, seed: int = GRAPH_SEED, nlabels: int = 5, nthreads: int = 0) -> np.ndarray:
    """uint8 label per edge, uniform in [0, nlabels), equal on both directions of a pair."""
    lib = _load()
    lab = np.empty(g.ne, dtype=np.uint8)
    rc = lib.syn_edge_labels(g.nv, g.row_ptr.ctypes.data, g.col.ctypes.data, seed, nlabels,
                             lab.ctypes.data, nthreads)
    if rc != 0:
        raise ValueError("bad label count")
    return lab


def sources(n: int, nv: int, seed: int = 1) -> np.ndarray:
    """n walk sources uniform in [0, nv)."""
    lib = _load()
    out = np.empty(n, dtype=np.int32)
    if lib.syn_sources(n, nv, seed, out.ctypes.data) != 0:
        raise ValueError("bad vertex count")
    return out


def schema(length: int, nlabels: int = 5, seed: int = 1) -> np.ndarray:
    """A MetaPath schema: length labels uniform in [0, nlabels)."""
    lib = _load()
    out = np.empty(length, dtype=np.uint8)
    if lib.syn_schema(length, nlabels, seed, out.ctypes.data) != 0:
        raise ValueError("bad schema")
    return out


def draw(seed: int, tag: int, i: int) -> int:
    """The i-th 64-bit value of stream (seed, tag); exposed for tests of the generator."""
    return int(_load().syn_draw(seed, tag, i))


def from_edges(nv: int, edges, symmetric: bool = False) -> Graph:
    """A small CSR graph from an explicit edge list (self-loops dropped, rows sorted, de-duplicated)."""
    adj = [set() for _ in range(nv)]
    for u, v in edges:
        if u == v:
            continue
        adj[u].add(v)
        if symmetric:
            adj[v].add(u)
    row_ptr = np.zeros(nv + 1, dtype=np.int64)
    for v in range(nv):
        row_ptr[v + 1] = row_ptr[v] + len(adj[v])
    col = np.array([x for v in range(nv) for x in sorted(adj[v])], dtype=np.int32)
    return Graph(row_ptr=row_ptr, col=col, name=f"edges-{nv}")


def vertex_sources(nv: int) -> np.ndarray:
    """One walk per vertex, in vertex order (the DeepWalk / Node2Vec source list)."""
    return np.arange(nv, dtype=np.int32)
