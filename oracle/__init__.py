"""ORACLE -- test infrastructure, not part of the product.

A plain single-threaded CPU walker (``oracle.c``) for the Gather-Move-Update
random-walk model of ThunderRW (Section 4.2, Algorithm 2), loaded through
ctypes.  Only the tests, the package's smoke check and the bench's
CPU-baseline leg may import this module.  It shares no code with the CUDA
library and never imports it.
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
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

DEEPWALK, DEEPWALK_WEIGHTED, PPR, NODE2VEC, METAPATH, NODE2VEC_WEIGHTED = 0, 1, 2, 3, 4, 5
OK, ERR_INVALID, ERR_OOM, ERR_REJECT_CAP = 0, -1, -2, -6
# Sampling methods of weighted DeepWalk (Section 2.3); DEFAULT is ALIAS.
SAMPLER_DEFAULT, SAMPLER_ITS, SAMPLER_REJ, SAMPLER_OREJ = 0, 1, 2, 3
ALGO_NAMES = {DEEPWALK: "deepwalk", DEEPWALK_WEIGHTED: "deepwalk_weighted", PPR: "ppr",
              NODE2VEC: "node2vec", METAPATH: "metapath", NODE2VEC_WEIGHTED: "node2vec_weighted"}


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-Wall", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Graph(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int64), ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
                ("H", ctypes.c_void_p), ("A_first", ctypes.c_void_p), ("A_second", ctypes.c_void_p),
                ("dead", ctypes.c_void_p), ("labels", ctypes.c_void_p), ("weights", ctypes.c_void_p),
                ("cdf", ctypes.c_void_p), ("pmax", ctypes.c_void_p)]


class _Params(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int32), ("walks_per_source", ctypes.c_int32), ("ppr_stop", ctypes.c_double),
                ("n2v_p", ctypes.c_double), ("n2v_q", ctypes.c_double), ("schema", ctypes.c_void_p),
                ("schema_len", ctypes.c_int32), ("endpoints_only", ctypes.c_int32),
                ("walk_offset", ctypes.c_int64), ("sampler", ctypes.c_int32), ("max_weight", ctypes.c_double)]


class _Stats(ctypes.Structure):
    _fields_ = [("moves", ctypes.c_int64), ("attempts", ctypes.c_int64), ("stop_len", ctypes.c_int64),
                ("stop_coin", ctypes.c_int64), ("stop_dead", ctypes.c_int64), ("stop_schema", ctypes.c_int64),
                ("sectors", ctypes.c_int64), ("out_bytes", ctypes.c_int64), ("checks", ctypes.c_int64),
                ("return_only", ctypes.c_int64)]


_WEIGHT_FN = ctypes.CFUNCTYPE(ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                              ctypes.c_int32, ctypes.c_int32, ctypes.c_int64)
_UPDATE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                              ctypes.c_int32, ctypes.c_int32, ctypes.c_int64)


def _bind(path: str):
    """Load a compiled oracle library and declare its signatures."""
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    lib.orc_philox4x32_10.argtypes = [vp, vp, vp]
    lib.orc_threshold.argtypes = [ctypes.c_double]
    lib.orc_threshold.restype = ctypes.c_uint64
    lib.orc_quantize_weight.argtypes = [ctypes.c_float]
    lib.orc_quantize_weight.restype = ctypes.c_int64
    lib.orc_alias_build.argtypes = [ctypes.c_int64, vp, vp, vp, vp]
    lib.orc_alias_build.restype = ctypes.c_int
    lib.orc_prepare_alias.argtypes = [ctypes.c_int64, vp, vp, vp, vp, vp, vp]
    lib.orc_prepare_alias.restype = ctypes.c_int
    lib.orc_prepare_its.argtypes = [ctypes.c_int64, vp, vp, vp]
    lib.orc_prepare_its.restype = ctypes.c_int
    lib.orc_prepare_rej.argtypes = [ctypes.c_int64, vp, vp, vp]
    lib.orc_prepare_rej.restype = ctypes.c_int
    lib.orc_rej_threshold.argtypes = [ctypes.c_uint32, ctypes.c_uint64]
    lib.orc_rej_threshold.restype = ctypes.c_uint64
    lib.orc_walk_custom.argtypes = [ctypes.POINTER(_Graph), ctypes.c_int32, ctypes.c_uint32, _WEIGHT_FN, _UPDATE_FN,
                                    vp, vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                    ctypes.c_int64, vp, vp, ctypes.POINTER(_Stats)]
    lib.orc_walk_custom.restype = ctypes.c_int
    lib.orc_walk.argtypes = [ctypes.POINTER(_Graph), ctypes.POINTER(_Params), vp, ctypes.c_int64,
                             ctypes.c_int32, ctypes.c_uint64, vp, vp, ctypes.POINTER(_Stats)]
    lib.orc_walk.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(_LIB_PATH)
    return _lib


def compile_variant(src_text: str, out_dir: str, name: str = "variant"):
    """Compile a modified copy of the oracle source (tests plant mistakes this
    way to show that the pins catch them) and return its bound library."""
    src = os.path.join(out_dir, name + ".c")
    so = os.path.join(out_dir, "lib" + name + ".so")
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-w", "-shared", "-fPIC", src, "-o", so, "-lm"])
    return _bind(so)


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def philox4x32_10(ctr, key, lib=None) -> np.ndarray:
    """One Philox4x32-10 block for a 4-word counter and a 2-word key."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    (lib or _load()).orc_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def threshold(t: float, lib=None) -> int:
    """floor(t * 2^32) clamped to [0, 2^32]."""
    return int((lib or _load()).orc_threshold(float(t)))


def quantize_weight(w: float, lib=None) -> int:
    """round-half-even(w * 2^16) clamped to [0, 2^32-1]; -1 for a negative or non-finite w."""
    return int((lib or _load()).orc_quantize_weight(float(w)))


@dataclass
class AliasTables:
    H: np.ndarray         # uint64[ne]: H[i] / 2^32 = chance of A_first[i]; 2^32 for a one-element bucket
    A_first: np.ndarray   # int32[ne]: local slot of the first element (always i)
    A_second: np.ndarray  # int32[ne]: local slot of the donor, -1 when absent
    dead: np.ndarray      # uint8[nv]: 1 when the row has edges but no positive integer weight


def alias_build(W, lib=None) -> tuple:
    """ALIAS initialisation of one row of integer weights -> (H, A_first, A_second, dead)."""
    W = np.ascontiguousarray(W, dtype=np.uint32)
    d = W.shape[0]
    H = np.zeros(d, dtype=np.uint64)
    A1 = np.zeros(d, dtype=np.int32)
    A2 = np.zeros(d, dtype=np.int32)
    dead = (lib or _load()).orc_alias_build(d, W.ctypes.data, H.ctypes.data, A1.ctypes.data, A2.ctypes.data)
    return H, A1, A2, int(dead)


def prepare_alias(row_ptr: np.ndarray, weights: np.ndarray, lib=None) -> AliasTables:
    """Algorithm 3 for ALIAS over every vertex."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    weights = np.ascontiguousarray(weights, dtype=np.float32)
    nv = row_ptr.shape[0] - 1
    ne = int(row_ptr[-1])
    H = np.zeros(ne, dtype=np.uint64)
    A1 = np.zeros(ne, dtype=np.int32)
    A2 = np.zeros(ne, dtype=np.int32)
    dead = np.zeros(nv, dtype=np.uint8)
    rc = (lib or _load()).orc_prepare_alias(nv, row_ptr.ctypes.data, weights.ctypes.data, H.ctypes.data,
                                   A1.ctypes.data, A2.ctypes.data, dead.ctypes.data)
    if rc != OK:
        raise ValueError("invalid edge weight")
    return AliasTables(H, A1, A2, dead)


def prepare_its(row_ptr: np.ndarray, weights: np.ndarray, lib=None) -> np.ndarray:
    """Algorithm 3 for ITS: the per-row prefix sums P' of the integer weights, uint64[ne]."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    weights = np.ascontiguousarray(weights, dtype=np.float32)
    cdf = np.zeros(int(row_ptr[-1]), dtype=np.uint64)
    if (lib or _load()).orc_prepare_its(row_ptr.shape[0] - 1, row_ptr.ctypes.data, weights.ctypes.data,
                                        cdf.ctypes.data) != OK:
        raise ValueError("invalid edge weight")
    return cdf


def prepare_rej(row_ptr: np.ndarray, weights: np.ndarray, lib=None) -> np.ndarray:
    """Algorithm 3 for REJ: p*_v, the largest integer weight of each row, uint32[nv]."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    weights = np.ascontiguousarray(weights, dtype=np.float32)
    pmax = np.zeros(row_ptr.shape[0] - 1, dtype=np.uint32)
    if (lib or _load()).orc_prepare_rej(row_ptr.shape[0] - 1, row_ptr.ctypes.data, weights.ctypes.data,
                                        pmax.ctypes.data) != OK:
        raise ValueError("invalid edge weight")
    return pmax


def rej_threshold(W: int, pstar: int, lib=None) -> int:
    """Acceptance threshold of a rejection dart: floor(W * 2^32 / p*), 2^32 once W >= p*."""
    return int((lib or _load()).orc_rej_threshold(int(W), int(pstar)))


@dataclass
class WalkResult:
    paths: np.ndarray     # int32[nwalks, max_len+1] (or [nwalks] for endpoints)
    lengths: np.ndarray   # int32[nwalks]: vertices per walk
    stats: dict
    status: int


def walk(row_ptr, col, algo: int, sources, max_len: int, seed: int, *, alias: Optional[AliasTables] = None,
         labels=None, ppr_stop: float = 0.0, n2v_p: float = 1.0, n2v_q: float = 1.0, schema=None,
         walks_per_source: int = 1, endpoints_only: bool = False, walk_offset: int = 0,
         sampler: int = SAMPLER_DEFAULT, weights=None, its=None, pmax=None, max_weight: float = 0.0,
         lib=None) -> WalkResult:
    """Run the oracle walker; returns paths, lengths, counters and the status code."""
    lib = lib or _load()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    sources = np.ascontiguousarray(sources, dtype=np.int32)
    keep = [row_ptr, col, sources]
    g = _Graph()
    g.nv = row_ptr.shape[0] - 1
    g.row_ptr = row_ptr.ctypes.data
    g.col = col.ctypes.data
    if alias is not None:
        g.H, g.A_first, g.A_second, g.dead = (alias.H.ctypes.data, alias.A_first.ctypes.data,
                                              alias.A_second.ctypes.data, alias.dead.ctypes.data)
    if labels is not None:
        labels = np.ascontiguousarray(labels, dtype=np.uint8)
        keep.append(labels)
        g.labels = labels.ctypes.data
    if weights is not None:
        weights = np.ascontiguousarray(weights, dtype=np.float32)
        keep.append(weights)
        g.weights = weights.ctypes.data
    if its is not None:
        its = np.ascontiguousarray(its, dtype=np.uint64)
        keep.append(its)
        g.cdf = its.ctypes.data
    if pmax is not None:
        pmax = np.ascontiguousarray(pmax, dtype=np.uint32)
        keep.append(pmax)
        g.pmax = pmax.ctypes.data
    p = _Params()
    p.algo = algo
    p.walks_per_source = walks_per_source
    p.ppr_stop = ppr_stop
    p.n2v_p = n2v_p
    p.n2v_q = n2v_q
    if schema is not None:
        schema = np.ascontiguousarray(schema, dtype=np.uint8)
        keep.append(schema)
        p.schema = schema.ctypes.data
        p.schema_len = schema.shape[0]
    p.endpoints_only = int(endpoints_only)
    p.walk_offset = walk_offset
    p.sampler = sampler
    p.max_weight = max_weight
    nwalks = sources.shape[0] * walks_per_source
    width = 1 if endpoints_only else max_len + 1
    paths = np.full((nwalks, width) if not endpoints_only else (nwalks,), -1, dtype=np.int32)
    lengths = np.zeros(nwalks, dtype=np.int32)
    st = _Stats()
    rc = lib.orc_walk(ctypes.byref(g), ctypes.byref(p), sources.ctypes.data, sources.shape[0], max_len, seed,
                      paths.ctypes.data, lengths.ctypes.data, ctypes.byref(st))
    stats = {name: getattr(st, name) for name, _ in _Stats._fields_}
    return WalkResult(paths, lengths, stats, rc)


NAIVE_SAMPLER, OREJ_SAMPLER = 0, 1


def walk_custom(row_ptr, col, sources, max_len: int, seed: int, *, sampler: int, weight=None, max_weight: int = 0,
                update=None, walks_per_source: int = 1, walk_offset: int = 0, lib=None) -> WalkResult:
    """A walk given by user functions (Section 4.3): sampler NAIVE_SAMPLER or
    OREJ_SAMPLER; weight(walk, length, cur, prev, dst, edge) -> int and
    max_weight (O-REJ, fixed point); update(walk, length, cur, prev, dst, edge)
    -> bool, called after each move with the query moved (true ends the walk)."""
    lib = lib or _load()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    sources = np.ascontiguousarray(sources, dtype=np.int32)
    g = _Graph()
    g.nv = row_ptr.shape[0] - 1
    g.row_ptr = row_ptr.ctypes.data
    g.col = col.ctypes.data
    wfn = _WEIGHT_FN((lambda u, *a: int(weight(*a))) if weight else 0)
    ufn = _UPDATE_FN((lambda u, *a: 1 if update(*a) else 0) if update else 0)
    nwalks = sources.shape[0] * walks_per_source
    paths = np.full((nwalks, max_len + 1), -1, dtype=np.int32)
    lengths = np.zeros(nwalks, dtype=np.int32)
    st = _Stats()
    rc = lib.orc_walk_custom(ctypes.byref(g), sampler, max_weight, wfn, ufn, None, sources.ctypes.data,
                             sources.shape[0], walks_per_source, max_len, seed, walk_offset, paths.ctypes.data,
                             lengths.ctypes.data, ctypes.byref(st))
    return WalkResult(paths, lengths, {name: getattr(st, name) for name, _ in _Stats._fields_}, rc)
