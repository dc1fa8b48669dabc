"""GB300-native random-walk engine: Python binding of libtrw.so (include/trw.h).

The binding only marshals arguments: every step of every walk runs in the
library's CUDA kernels.  Arrays may be numpy (host) or torch tensors (host or
CUDA).  There is no CPU fallback: importing works without a GPU, but every
call that needs one raises when the CUDA library or device is missing.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

from . import _build

__all__ = ["TRWError", "Graph", "Server", "load_library", "build", "DEEPWALK", "DEEPWALK_WEIGHTED", "PPR",
           "NODE2VEC", "METAPATH", "KERNEL_AUTO", "KERNEL_PLAIN", "KERNEL_PERSISTENT", "OUT_PATHS",
           "OUT_ENDPOINTS", "philox_device"]

DEEPWALK, DEEPWALK_WEIGHTED, PPR, NODE2VEC, METAPATH, NODE2VEC_WEIGHTED = 0, 1, 2, 3, 4, 5
KERNEL_AUTO, KERNEL_PLAIN, KERNEL_PERSISTENT, KERNEL_BSP = 0, 1, 2, 3
OUT_PATHS, OUT_ENDPOINTS, OUT_COMPACT = 0, 1, 2
PREP_ALIAS = 1
PREP_LABEL_INDEX = 2
LABEL_INDEX_MAX_LABELS = 30
PREP_NEIGHBOR_HASH = 4
PREP_ROW_RECORDS = 8
PREP_ITS = 16
PREP_REJ = 32
PREP_ITS_GUIDE = 64
PREP_ALL = (PREP_ALIAS | PREP_LABEL_INDEX | PREP_NEIGHBOR_HASH | PREP_ROW_RECORDS | PREP_ITS | PREP_REJ |
            PREP_ITS_GUIDE)
# Sampling method of weighted DeepWalk (Section 2.3): DEFAULT is ALIAS.
SAMPLER_DEFAULT, SAMPLER_ITS, SAMPLER_REJ, SAMPLER_OREJ = 0, 1, 2, 3
MAX_SCHEMA = 16
MAX_BATCH = 64

OK, PENDING = 0, 1
ERR_STOPPED, ERR_IO = -10, -11
_STREAM_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                              ctypes.c_void_p)
STATUS_NAMES = {0: "OK", 1: "PENDING", -1: "ERR_INVALID", -2: "ERR_OOM", -3: "ERR_NOT_PREPARED", -4: "ERR_CUDA",
                -5: "ERR_TIMEOUT", -6: "ERR_REJECT_CAP", -7: "ERR_BUSY", -8: "ERR_NOT_FOUND", -9: "ERR_INTERNAL"}

ALGOS = {"deepwalk": DEEPWALK, "deepwalk_weighted": DEEPWALK_WEIGHTED, "ppr": PPR, "node2vec": NODE2VEC,
         "metapath": METAPATH, "node2vec_weighted": NODE2VEC_WEIGHTED}


class TRWError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class _Params(ctypes.Structure):
    _fields_ = [("ppr_stop", ctypes.c_double), ("n2v_p", ctypes.c_double), ("n2v_q", ctypes.c_double),
                ("schema", ctypes.c_void_p), ("schema_len", ctypes.c_int32), ("out_mode", ctypes.c_uint32),
                ("walks_per_source", ctypes.c_int32), ("sampler", ctypes.c_int32), ("walk_offset", ctypes.c_int64),
                ("max_weight", ctypes.c_double)]


class Tuning(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("coop_degree", ctypes.c_int32), ("search_degree", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Stats(ctypes.Structure):
    _fields_ = [("walks", ctypes.c_int64), ("moves", ctypes.c_int64), ("kernel_ms", ctypes.c_double),
                ("grid_blocks", ctypes.c_int32), ("block_threads", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("launches", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServeConfig(ctypes.Structure):
    _fields_ = [("max_inflight_walks", ctypes.c_int64), ("max_inflight_bytes", ctypes.c_int64),
                ("max_requests", ctypes.c_int32), ("idle_timeout_us", ctypes.c_int32)]


_lib = None

# Every function the header declares, with its ctypes signature.
_VP = ctypes.c_void_p
_SIGS = {
    "trw_params_default": (None, [_VP]),
    "trw_graph_load": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, _VP, _VP, _VP, _VP, ctypes.c_uint32, _VP]),
    "trw_graph_free": (None, [_VP]),
    "trw_prepare": (ctypes.c_int, [_VP, ctypes.c_uint32]),
    "trw_walk": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, _VP,
                                _VP]),
    "trw_walk_ex": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, _VP,
                                   _VP, ctypes.c_int, _VP, ctypes.c_int]),
    "trw_sync": (ctypes.c_int, [_VP, _VP]),
    "trw_walk_batch": (ctypes.c_int, [_VP, ctypes.c_int32, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP,
                                      ctypes.c_int]),
    "trw_walk_batch_noalloc": (ctypes.c_int, [_VP, ctypes.c_int32, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "trw_plan_create": (ctypes.c_int, [_VP, ctypes.c_int32, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "trw_plan_set_seed": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_uint64]),
    "trw_plan_launch": (ctypes.c_int, [_VP, _VP]),
    "trw_plan_sync": (ctypes.c_int, [_VP, _VP]),
    "trw_plan_destroy": (None, [_VP]),
    "trw_get_tuning": (ctypes.c_int, [_VP, _VP]),
    "trw_set_tuning": (ctypes.c_int, [_VP, _VP]),
    "trw_autotune": (ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_int32, _VP]),
    "trw_last_stats": (ctypes.c_int, [_VP, _VP]),
    "trw_graph_get_view": (ctypes.c_int, [_VP, _VP]),
    "trw_graph_nv": (ctypes.c_int64, [_VP]),
    "trw_graph_ne": (ctypes.c_int64, [_VP]),
    "trw_graph_device_bytes": (ctypes.c_int64, [_VP]),
    "trw_debug_alias": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "trw_debug_label_index": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "trw_debug_sampler_tables": (ctypes.c_int, [_VP, _VP, _VP]),
    "trw_debug_its_records": (ctypes.c_int, [_VP, _VP]),
    "trw_debug_row_records": (ctypes.c_int, [_VP, _VP]),
    "trw_debug_is_neighbor": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, _VP]),
    "trw_debug_philox": (ctypes.c_int, [_VP, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint32, _VP]),
    "trw_debug_fail_allocs": (None, [ctypes.c_int64]),
    "trw_debug_pretend_device": (None, [ctypes.c_int32]),
    "trw_serve_config_default": (None, [_VP]),
    "trw_serve_create": (ctypes.c_int, [_VP, _VP, _VP]),
    "trw_serve_submit": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, ctypes.c_int64, ctypes.c_int32,
                                        ctypes.c_uint64, _VP, _VP, _VP]),
    "trw_serve_order_after": (ctypes.c_int, [_VP, _VP]),
    "trw_serve_poll": (ctypes.c_int, [_VP, ctypes.c_uint64]),
    "trw_serve_reap": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int32, _VP]),
    "trw_serve_trace": (ctypes.c_int, [_VP, ctypes.c_uint64, _VP]),
    "trw_serve_drain": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "trw_serve_destroy": (None, [_VP]),
    "trw_walk_stream": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                       ctypes.c_int64, _VP, _VP]),
    "trw_walk_to_file": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                        ctypes.c_char_p, ctypes.c_char_p]),
    "trw_gather_ceiling": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _VP, _VP]),
    "trw_last_error": (ctypes.c_char_p, []),
}


def build(force: bool = False) -> str:
    """Compile libtrw.so for sm_103a (nvcc) if it is missing or stale."""
    return _build.build(force=force)


def load_library(path: Optional[str] = None):
    """Load libtrw.so (building it first if missing).  Raises if it cannot be built or loaded."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _build.LIB
    if path is None and (not os.path.exists(p) or _build.stale()):
        _build.build()
    try:
        lib = ctypes.CDLL(p)
    except OSError as e:
        raise RuntimeError(f"cannot load the CUDA walk library {p}: {e}") from e
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _check(status: int, what: str = ""):
    if status != OK:
        msg = load_library().trw_last_error()
        raise TRWError(status, (what + ": " if what else "") + (msg.decode() if msg else ""))


# ------------------------------------------------------------ array helpers

def _torch():
    import torch
    return torch


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x) -> int:
    if x is None:
        return 0
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"unsupported array type {type(x)}")


def _as_host(x, dtype):
    if _is_torch(x):
        x = x.detach().cpu().numpy()
    return np.ascontiguousarray(x, dtype=dtype)


def _current_stream_handle() -> int:
    """The caller's current CUDA stream as a cudaStream_t (1: the legacy
    default stream), without building a torch Stream object where torch
    exposes the raw handle."""
    torch = _torch()
    raw = getattr(torch._C, "_cuda_getCurrentRawStream", None)
    h = raw(torch.cuda.current_device()) if raw is not None else torch.cuda.current_stream().cuda_stream
    return h or 1


def _is_cuda(x) -> bool:
    return _is_torch(x) and x.is_cuda


def _stream_arg(stream, *arrays) -> int:
    """The cudaStream_t to pass: an explicit handle, else torch's current stream
    when CUDA tensors are involved (handle 0, torch's default stream, is passed
    as cudaStreamLegacy), else 0 for the graph's own stream."""
    if stream is not None:
        if hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        return int(stream) or 1
    if any(_is_cuda(a) for a in arrays):
        return _current_stream_handle()
    return 0


def _params(algo: int, ppr_stop: float, n2v_p: float, n2v_q: float, schema, walks_per_source: int,
            endpoints: bool, walk_offset: int, sampler: int = SAMPLER_DEFAULT, max_weight: float = 0.0):
    p = _Params()
    p.sampler = sampler
    p.max_weight = max_weight
    p.ppr_stop = ppr_stop
    p.n2v_p = n2v_p
    p.n2v_q = n2v_q
    keep = None
    if schema is not None:
        keep = np.ascontiguousarray(_as_host(schema, np.uint8))
        p.schema = keep.ctypes.data
        p.schema_len = keep.shape[0]
    p.out_mode = OUT_ENDPOINTS if endpoints else OUT_PATHS
    p.walks_per_source = walks_per_source
    p.walk_offset = walk_offset
    return p, keep


@dataclass
class WalkOutput:
    paths: object     # int32 [nwalks, max_len+1] or [nwalks] (numpy or torch, like the sources)
    lengths: object   # int32 [nwalks]


class Graph:
    """A CSR graph resident on the current CUDA device (trw_graph_load)."""

    def __init__(self, row_ptr, col, weights=None, labels=None, check: bool = True):
        lib = load_library()
        rp = _as_host(row_ptr, np.int64)
        cl = _as_host(col, np.int32)
        w = None if weights is None else _as_host(weights, np.float32)
        lab = None if labels is None else _as_host(labels, np.uint8)
        for name, a in (("weights", w), ("labels", lab)):
            if a is not None and a.shape != cl.shape:
                raise ValueError(f"{name} has {a.shape[0]} entries for {cl.shape[0]} edges")
        h = ctypes.c_void_p(0)
        st = lib.trw_graph_load(rp.shape[0] - 1, cl.shape[0], rp.ctypes.data, cl.ctypes.data,
                                0 if w is None else w.ctypes.data, 0 if lab is None else lab.ctypes.data,
                                1 if check else 0, ctypes.byref(h))
        _check(st, "trw_graph_load")
        self._h = h
        self.nv = int(rp.shape[0] - 1)
        self.ne = int(cl.shape[0])
        self.has_weights = w is not None
        self.has_labels = lab is not None

    @classmethod
    def from_synth(cls, g):
        return cls(g.row_ptr, g.col, g.weights, g.labels)

    @property
    def handle(self):
        return self._h

    def free(self):
        if getattr(self, "_h", None) and self._h.value:
            load_library().trw_graph_free(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def prepare(self, what: int = PREP_ALIAS):
        """trw_prepare: PREP_ALIAS (weighted DeepWalk tables), PREP_LABEL_INDEX
        (MetaPath label index), PREP_NEIGHBOR_HASH (Node2Vec IsNeighbor) and/or
        PREP_ROW_RECORDS (one read per NAIVE move or O-REJ candidate), PREP_ITS and
        PREP_REJ (the tables of weighted DeepWalk's ITS and REJ samplers) and
        PREP_ITS_GUIDE (guided ITS records: the same ITS walks in about two reads a move)."""
        _check(load_library().trw_prepare(self._h, what), "trw_prepare")

    def device_bytes(self) -> int:
        return int(load_library().trw_graph_device_bytes(self._h))

    # -------------------------------------------------------------- walks
    def walk(self, algo: int, sources, max_len: int, seed: int, *, ppr_stop: float = 0.2, n2v_p: float = 1.0,
             n2v_q: float = 1.0, schema=None, walks_per_source: int = 1, endpoints: bool = False,
             walk_offset: int = 0, kernel: int = KERNEL_AUTO, out_paths=None, out_lengths=None, stream=None,
             sync: bool = True, sampler: int = SAMPLER_DEFAULT, max_weight: float = 0.0,
             compact: bool = False) -> WalkOutput:
        """trw_walk_ex.  Outputs follow the sources: numpy for host sources, CUDA
        tensors for CUDA sources, unless out_paths / out_lengths are given.
        sampler / max_weight choose weighted DeepWalk's sampling method.
        compact: TRW_OUT_COMPACT, paths is the walks' vertices one after the
        other (trimmed to the sum of the lengths when the call allocates it)."""
        lib = load_library()
        algo = ALGOS.get(algo, algo) if isinstance(algo, str) else algo
        p, keep = _params(algo, ppr_stop, n2v_p, n2v_q, schema, walks_per_source, endpoints, walk_offset, sampler,
                          max_weight)
        if compact:
            p.out_mode = OUT_COMPACT
        if _is_torch(sources):
            src = sources if sources.dtype == _torch().int32 else sources.to(_torch().int32)
            src = src.contiguous()
        else:
            src = np.ascontiguousarray(sources, dtype=np.int32)
        n = int(src.shape[0])
        nwalks = n * walks_per_source
        shape = (nwalks,) if endpoints else ((nwalks * (max_len + 1),) if compact else (nwalks, max_len + 1))
        trim = compact and out_paths is None
        if out_paths is None:
            out_paths = (_torch().empty(shape, dtype=_torch().int32, device=src.device) if _is_cuda(src)
                         else np.empty(shape, dtype=np.int32))
        if out_lengths is None:
            out_lengths = (_torch().empty(nwalks, dtype=_torch().int32, device=src.device) if _is_cuda(src)
                           else np.empty(nwalks, dtype=np.int32))
        st = lib.trw_walk_ex(self._h, algo, ctypes.byref(p), _ptr(src), n, max_len, seed & ((1 << 64) - 1),
                             _ptr(out_paths), _ptr(out_lengths), kernel, _stream_arg(stream, src, out_paths, out_lengths),
                             1 if sync else 0)
        _check(st, "trw_walk")
        if trim and sync:
            total = int(out_lengths.sum().item()) if _is_torch(out_lengths) else int(out_lengths.sum())
            out_paths = out_paths[:total]
        return WalkOutput(out_paths, out_lengths)

    def walk_stream(self, algo: int, sources, max_len: int, seed: int, consumer, *, slice_walks: int = 1 << 20,
                    ppr_stop: float = 0.2, n2v_p: float = 1.0, n2v_q: float = 1.0, schema=None,
                    walks_per_source: int = 1, endpoints: bool = False, walk_offset: int = 0,
                    sampler: int = SAMPLER_DEFAULT, max_weight: float = 0.0) -> int:
        """trw_walk_stream: consumer(first_walk, paths, lengths) receives each slice
        as numpy views of pinned host memory, valid during the call only (paths
        [n, max_len + 1], or [n] with endpoints); a true return value stops the
        stream (TRWError ERR_STOPPED).  The consumer must not walk this graph
        (the graph is locked while it runs).  Returns the moves of the batch."""
        lib = load_library()
        algo = ALGOS.get(algo, algo) if isinstance(algo, str) else algo
        p, keep = _params(algo, ppr_stop, n2v_p, n2v_q, schema, walks_per_source, endpoints, walk_offset, sampler,
                          max_weight)
        src = sources if _is_cuda(sources) else np.ascontiguousarray(_as_host(sources, np.int32))
        if _is_cuda(src):
            src = src.to(_torch().int32).contiguous()
            _torch().cuda.current_stream().synchronize()
        row = 1 if endpoints else max_len + 1
        raised = []

        def cb(_user, first, n, paths, lengths):
            try:
                pa = np.ctypeslib.as_array(ctypes.cast(paths, ctypes.POINTER(ctypes.c_int32)), shape=(n * row,))
                la = np.ctypeslib.as_array(ctypes.cast(lengths, ctypes.POINTER(ctypes.c_int32)), shape=(n,))
                stop = consumer(int(first), pa if endpoints else pa.reshape(n, row), la)
                return 1 if stop else 0
            except BaseException as e:  # re-raised after the call
                raised.append(e)
                return 1

        fn = _STREAM_FN(cb)
        st = lib.trw_walk_stream(self._h, algo, ctypes.byref(p), _ptr(src), int(src.shape[0]), max_len,
                                 seed & ((1 << 64) - 1), slice_walks, fn, None)
        if raised:
            raise raised[0]
        _check(st, "trw_walk_stream")
        return int(self.last_stats()["moves"])

    def walk_to_file(self, algo: int, sources, max_len: int, seed: int, paths_file: str, lengths_file: str, *,
                     ppr_stop: float = 0.2, n2v_p: float = 1.0, n2v_q: float = 1.0, schema=None,
                     walks_per_source: int = 1, endpoints: bool = False, walk_offset: int = 0,
                     sampler: int = SAMPLER_DEFAULT, max_weight: float = 0.0) -> int:
        """trw_walk_to_file: the vertices of every walk, walk after walk, to
        paths_file and the int32 lengths to lengths_file.  Returns the moves."""
        lib = load_library()
        algo = ALGOS.get(algo, algo) if isinstance(algo, str) else algo
        p, keep = _params(algo, ppr_stop, n2v_p, n2v_q, schema, walks_per_source, endpoints, walk_offset, sampler,
                          max_weight)
        src = sources if _is_cuda(sources) else np.ascontiguousarray(_as_host(sources, np.int32))
        if _is_cuda(src):
            src = src.to(_torch().int32).contiguous()
            _torch().cuda.current_stream().synchronize()
        _check(lib.trw_walk_to_file(self._h, algo, ctypes.byref(p), _ptr(src), int(src.shape[0]), max_len,
                                    seed & ((1 << 64) - 1), os.fsencode(paths_file), os.fsencode(lengths_file)),
               "trw_walk_to_file")
        return int(self.last_stats()["moves"])

    def sync(self, stream=None):
        """Wait for the stream (default: torch's current stream) and collect the device status."""
        sa = _stream_arg(stream) if stream is not None else (int(_torch().cuda.current_stream().cuda_stream) or 1)
        _check(load_library().trw_sync(self._h, sa), "trw_sync")

    def _batch_args(self, requests: Sequence[dict], outputs=None):
        """ctypes arrays of a mixed batch; outputs allocated as CUDA tensors
        unless given as (paths, lengths) pairs, one per request."""
        torch = _torch()
        nreq = len(requests)
        if not 1 <= nreq <= MAX_BATCH:
            raise ValueError(f"1..{MAX_BATCH} requests")
        algos = (ctypes.c_int * nreq)()
        params = (_Params * nreq)()
        srcs = (ctypes.c_void_p * nreq)()
        ns = (ctypes.c_int64 * nreq)()
        lens = (ctypes.c_int32 * nreq)()
        seeds = (ctypes.c_uint64 * nreq)()
        outs = (ctypes.c_void_p * nreq)()
        outl = (ctypes.c_void_p * nreq)()
        keep, results = [], []
        for i, r in enumerate(requests):
            algo = r["algo"]
            algo = ALGOS.get(algo, algo) if isinstance(algo, str) else algo
            wps = r.get("walks_per_source", 1)
            ep = r.get("endpoints", False)
            p, k = _params(algo, r.get("ppr_stop", 0.2), r.get("n2v_p", 1.0), r.get("n2v_q", 1.0), r.get("schema"),
                           wps, ep, r.get("walk_offset", 0), r.get("sampler", SAMPLER_DEFAULT),
                           r.get("max_weight", 0.0))
            keep.append(k)
            src = r["sources"]
            if not _is_cuda(src):
                src = torch.as_tensor(np.ascontiguousarray(src, dtype=np.int32)).cuda()
            src = src.to(torch.int32).contiguous()
            keep.append(src)
            n = int(src.shape[0])
            L = int(r["max_len"])
            shape = (n * wps,) if ep else (n * wps, L + 1)
            if outputs is not None:
                op, ol = outputs[i]
                if tuple(op.shape) != shape or tuple(ol.shape) != (n * wps,) or not (_is_cuda(op) and _is_cuda(ol)):
                    raise ValueError(f"request {i}: outputs must be CUDA tensors of shapes {shape} and {(n * wps,)}")
            else:
                op = torch.empty(shape, dtype=torch.int32, device=src.device)
                ol = torch.empty(n * wps, dtype=torch.int32, device=src.device)
            algos[i], params[i], srcs[i], ns[i], lens[i] = algo, p, src.data_ptr(), n, L
            seeds[i] = int(r["seed"]) & ((1 << 64) - 1)
            outs[i], outl[i] = op.data_ptr(), ol.data_ptr()
            results.append(WalkOutput(op, ol))
        return (nreq, algos, params, srcs, ns, lens, seeds, outs, outl), keep, results

    def walk_batch(self, requests: Sequence[dict], stream=None, sync: bool = True, outputs=None):
        """One persistent launch over a mixed batch.  Each request is a dict with
        algo, sources (CUDA tensor), max_len, seed and optional parameters; outputs
        are allocated as CUDA tensors (or taken from `outputs`, one (paths,
        lengths) pair per request) and returned as a list of WalkOutput."""
        args, keep, results = self._batch_args(requests, outputs)
        st = load_library().trw_walk_batch(self._h, *args, _stream_arg(stream, *[k for k in keep if _is_torch(k)]),
                                           1 if sync else 0)
        _check(st, "trw_walk_batch")
        return results

    def plan(self, requests: Sequence[dict]) -> "Plan":
        """The mixed batch captured once as a CUDA graph (trw_plan_create)."""
        return Plan(self, requests)

    def tuning(self) -> dict:
        t = Tuning()
        _check(load_library().trw_get_tuning(self._h, ctypes.byref(t)))
        return t.as_dict()

    def set_tuning(self, **kw):
        t = Tuning()
        _check(load_library().trw_get_tuning(self._h, ctypes.byref(t)))
        for k, v in kw.items():
            setattr(t, k, v)
        _check(load_library().trw_set_tuning(self._h, ctypes.byref(t)), "trw_set_tuning")

    def autotune(self, algo: int, max_len: int = 10, **kw) -> dict:
        p, keep = _params(algo, kw.get("ppr_stop", 0.2), kw.get("n2v_p", 1.0), kw.get("n2v_q", 1.0),
                          kw.get("schema"), 1, kw.get("endpoints", False), 0, kw.get("sampler", SAMPLER_DEFAULT),
                          kw.get("max_weight", 0.0))
        t = Tuning()
        _check(load_library().trw_autotune(self._h, algo, ctypes.byref(p), max_len, ctypes.byref(t)), "trw_autotune")
        return t.as_dict()

    def last_stats(self) -> dict:
        s = Stats()
        _check(load_library().trw_last_stats(self._h, ctypes.byref(s)))
        return s.as_dict()

    def debug_alias(self):
        H = np.empty(self.ne, dtype=np.uint32)
        a = np.empty(self.ne, dtype=np.int32)
        b = np.empty(self.ne, dtype=np.int32)
        _check(load_library().trw_debug_alias(self._h, H.ctypes.data, a.ctypes.data, b.ctypes.data), "trw_debug_alias")
        return H, a, b

    def debug_label_index(self):
        """(stride, vertex records [nv, stride], edge records [ne, stride]) of
        the MetaPath label index, or None when it is not prepared."""
        lib = load_library()
        st = ctypes.c_int32(0)
        _check(lib.trw_debug_label_index(self._h, ctypes.byref(st), None, None), "trw_debug_label_index")
        if st.value == 0:
            return None
        v = np.empty((self.nv, st.value), dtype=np.int32)
        e = np.empty((self.ne, st.value), dtype=np.int32)
        _check(lib.trw_debug_label_index(self._h, ctypes.byref(st), v.ctypes.data, e.ctypes.data),
               "trw_debug_label_index")
        return st.value, v, e

    def debug_sampler_tables(self, its: bool = True, rej: bool = True):
        """(ITS prefix sums uint64[ne] or None, REJ bounds uint32[nv] or None) from the device."""
        cdf = np.empty(self.ne, dtype=np.uint64) if its else None
        pm = np.empty(self.nv, dtype=np.uint32) if rej else None
        _check(load_library().trw_debug_sampler_tables(self._h, None if cdf is None else cdf.ctypes.data,
                                                        None if pm is None else pm.ctypes.data),
               "trw_debug_sampler_tables")
        return cdf, pm

    def debug_its_records(self) -> np.ndarray:
        """Guided ITS records as uint32 [ne, 8]: U low/high, destination, its row
        offset and degree, the cell's first and last candidates, 0."""
        out = np.empty((self.ne, 8), dtype=np.uint32)
        _check(load_library().trw_debug_its_records(self._h, out.ctypes.data), "trw_debug_its_records")
        return out

    def debug_row_records(self) -> np.ndarray:
        """Row records as int32 [ne, 4]: destination, its row offset and degree,
        and aux: the integer weight on a weighted graph, else the position of
        the source in the destination's row (-1: none)."""
        out = np.empty((self.ne, 4), dtype=np.int32)
        _check(load_library().trw_debug_row_records(self._h, out.ctypes.data), "trw_debug_row_records")
        return out

    def debug_is_neighbor(self, u, v) -> np.ndarray:
        """IsNeighbor(v[i], u[i]) as the walk kernels evaluate it (bool array)."""
        u = np.ascontiguousarray(u, dtype=np.int32)
        v = np.ascontiguousarray(v, dtype=np.int32)
        out = np.empty(u.shape[0], dtype=np.uint8)
        _check(load_library().trw_debug_is_neighbor(self._h, u.ctypes.data, v.ctypes.data, u.shape[0],
                                                    out.ctypes.data), "trw_debug_is_neighbor")
        return out.astype(bool)


def gather_ceiling(table_bytes: int, record_bytes: int = 16, hops: int = 80, chains: int = 1) -> dict:
    """Random dependent-load rate of this GPU (trw_gather_ceiling)."""
    lps = ctypes.c_double(0)
    ms = ctypes.c_double(0)
    _check(load_library().trw_gather_ceiling(table_bytes, record_bytes, hops, chains, ctypes.byref(lps),
                                             ctypes.byref(ms)), "trw_gather_ceiling")
    return {"loads_per_s": lps.value, "kernel_ms": ms.value, "table_bytes": table_bytes,
            "record_bytes": record_bytes, "hops": hops, "chains": chains}


def philox_device(ctr, key0: int, key1: int) -> np.ndarray:
    """Philox4x32-10 blocks computed by the device code (for tests)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.empty_like(c)
    _check(load_library().trw_debug_philox(c.ctypes.data, c.shape[0], key0, key1, out.ctypes.data), "philox")
    return out


def fail_allocs(after: int) -> None:
    """Test hook (trw_debug_fail_allocs): after the next `after` device or
    pinned allocations of the library every later one fails as out of memory;
    a negative `after` turns the failures off."""
    load_library().trw_debug_fail_allocs(int(after))


def pretend_device(device: int) -> None:
    """Test hook (trw_debug_pretend_device): the library's device checks
    compare graphs with `device` instead of the current device (negative:
    the current device again).  Calls refuse; nothing launches elsewhere."""
    load_library().trw_debug_pretend_device(int(device))


class Plan:
    """A mixed batch captured as a CUDA graph (trw_plan_*): every launch()
    re-walks the batch into the same output tensors (.outputs)."""

    def __init__(self, graph: Graph, requests: Sequence[dict]):
        lib = load_library()
        args, self._keep, self.outputs = graph._batch_args(requests)
        _torch().cuda.current_stream().synchronize()  # sources copied on torch's stream
        self.graph = graph
        h = ctypes.c_void_p(0)
        _check(lib.trw_plan_create(graph._h, *args, ctypes.byref(h)), "trw_plan_create")
        self._h = h

    def launch(self, stream=None):
        _check(load_library().trw_plan_launch(self._h, _stream_arg(stream)), "trw_plan_launch")

    def sync(self) -> int:
        """Waits for the last launch; returns its moves (raises on a device error)."""
        moves = ctypes.c_int64(0)
        _check(load_library().trw_plan_sync(self._h, ctypes.byref(moves)), "trw_plan_sync")
        return moves.value

    def set_seed(self, request: int, seed: int):
        _check(load_library().trw_plan_set_seed(self._h, request, int(seed) & ((1 << 64) - 1)), "trw_plan_set_seed")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load_library().trw_plan_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching serving loop over a resident graph (trw_serve_*)."""

    def __init__(self, graph: Graph, max_inflight_walks: int = 0, max_inflight_bytes: int = 0,
                 max_requests: int = 0, idle_timeout_us: int = 0):
        lib = load_library()
        cfg = ServeConfig()
        lib.trw_serve_config_default(ctypes.byref(cfg))
        if max_inflight_walks:
            cfg.max_inflight_walks = max_inflight_walks
        if max_inflight_bytes:
            cfg.max_inflight_bytes = max_inflight_bytes
        if max_requests:
            cfg.max_requests = max_requests
        if idle_timeout_us:
            cfg.idle_timeout_us = idle_timeout_us
        h = ctypes.c_void_p(0)
        _check(lib.trw_serve_create(graph.handle, ctypes.byref(cfg), ctypes.byref(h)), "trw_serve_create")
        self._h = h
        self.graph = graph
        self._keep = {}
        self._reap_bufs = {}

    def submit(self, algo: int, sources, max_len: int, seed: int, out_paths, out_lengths, *, ppr_stop: float = 0.2,
               n2v_p: float = 1.0, n2v_q: float = 1.0, schema=None, walks_per_source: int = 1,
               endpoints: bool = False, walk_offset: int = 0, sampler: int = SAMPLER_DEFAULT,
               max_weight: float = 0.0) -> int:
        """Queue a request; raises TRWError(ERR_BUSY) when it cannot be admitted now."""
        lib = load_library()
        p, keep = _params(algo, ppr_stop, n2v_p, n2v_q, schema, walks_per_source, endpoints, walk_offset, sampler,
                          max_weight)
        src = sources if _is_torch(sources) else np.ascontiguousarray(sources, dtype=np.int32)
        if _is_cuda(src) or _is_cuda(out_paths) or _is_cuda(out_lengths):
            # the server runs on its own streams: work queued on the caller's
            # stream for these buffers (allocation, fills) must finish before
            # the request becomes visible -- ordered on the device, not waited for
            _check(lib.trw_serve_order_after(self._h, _current_stream_handle()), "trw_serve_order_after")
        rid = ctypes.c_uint64(0)
        st = lib.trw_serve_submit(self._h, algo, ctypes.byref(p), _ptr(src), int(src.shape[0]), max_len,
                                  seed & ((1 << 64) - 1), _ptr(out_paths), _ptr(out_lengths), ctypes.byref(rid))
        _check(st, "trw_serve_submit")
        self._keep[rid.value] = (src, out_paths, out_lengths)  # device sources are read after submit returns
        return rid.value

    def poll(self, rid: int) -> int:
        """OK (0) when done, PENDING (1) while running; raises on a request error."""
        st = load_library().trw_serve_poll(self._h, rid)
        if st == PENDING:
            return PENDING
        self._keep.pop(rid, None)
        _check(st, f"request {rid}")
        return OK

    def reap(self, max_requests: int = 256):
        """Finished requests, oldest first, as (request id, status) pairs (status 0
        is OK, else the request's error status); empty when none has finished."""
        bufs = self._reap_bufs.get(max_requests)
        if bufs is None:  # kept per size: a poll loop reaps often
            bufs = self._reap_bufs[max_requests] = ((ctypes.c_uint64 * max_requests)(),
                                                    (ctypes.c_int32 * max_requests)(), ctypes.c_int32(0))
        ids, sts, n = bufs
        _check(load_library().trw_serve_reap(self._h, ids, sts, max_requests, ctypes.byref(n)), "trw_serve_reap")
        out = []
        for i in range(n.value):
            self._keep.pop(int(ids[i]), None)
            out.append((int(ids[i]), int(sts[i])))
        return out

    def trace(self, rid: int) -> dict:
        """Device timeline of a request (ns on the device clock; 0 = not yet):
        admitted by the dispatcher, first walks started, last walk finished."""
        t = (ctypes.c_uint64 * 3)()
        _check(load_library().trw_serve_trace(self._h, rid, t), "trw_serve_trace")
        return {"admit_ns": int(t[0]), "first_ns": int(t[1]), "done_ns": int(t[2])}

    def drain(self, timeout_ms: int = 60000):
        _check(load_library().trw_serve_drain(self._h, timeout_ms), "trw_serve_drain")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load_library().trw_serve_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
