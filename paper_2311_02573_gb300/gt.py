"""Python binding of the C ABI in include/gt.h (argument marshalling only).

Every step of the search runs in the CUDA library ``_lib/libgt.so``; there
is no Python or CPU fallback.  Inputs may be numpy arrays (host memory) or
torch tensors (host or CUDA); float32, C-contiguous, row-major.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

GT_F32, GT_BF16, GT_FP8 = 0, 1, 2
DTYPES = {"f32": GT_F32, "bf16": GT_BF16, "fp8": GT_FP8}
POOLING = {"sum": 0, "max": 1, "maxmin": 2}
LAYOUTS = {"tree": 0, "prefix": 1}
STATUS = {0: "GT_OK", 1: "GT_EINVAL", 2: "GT_EDOMAIN", 3: "GT_ENOMEM", 4: "GT_ECUDA",
          5: "GT_ETIMEOUT", 6: "GT_EOVERFLOW", 7: "GT_EBUSY"}

_c_i64, _c_i32, _c_u32, _c_p, _c_f64 = (ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32,
                                        ctypes.c_void_p, ctypes.c_double)


class BuildOpts(ctypes.Structure):
    _fields_ = [("stream", _c_p), ("perm", _c_p), ("capacity", _c_i64), ("formats", _c_u32),
                ("pooling", _c_i32), ("layout", _c_i32), ("prefix_level", _c_i32)]


class QueryStats(ctypes.Structure):
    _fields_ = [("tests", _c_i64), ("dense_tests", _c_i64), ("gathered_tests", _c_i64),
                ("rechecks", _c_i64), ("results", _c_i64), ("micro_batches", _c_i64),
                ("retries", _c_i64), ("cutover", _c_i32), ("levels", _c_i32),
                ("level_tests", _c_i64 * 64), ("gathered_bytes", _c_f64),
                ("launches", _c_i64), ("level_launches", _c_i64),
                ("kernel_ms", ctypes.c_float * 8), ("refines", _c_i64),
                ("graph_captures", _c_i64), ("graph_replays", _c_i64)]
    KERNELS = ("levels", "leaf", "dense", "recheck", "csr", "prep", "bucket")

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_
             if k not in ("level_tests", "kernel_ms")}
        d["level_tests"] = list(self.level_tests)[: max(self.levels, 0)]
        d["kernel_ms"] = {k: float(self.kernel_ms[i]) for i, k in enumerate(self.KERNELS)}
        return d


class QueryOpts(ctypes.Structure):
    _fields_ = [("stream", _c_p), ("dtype", _c_i32), ("cutover", _c_i32),
                ("max_batch", _c_i64), ("scratch_bytes", _c_i64),
                ("results_on_device", _c_i32), ("timing", _c_i32),
                ("stats", ctypes.POINTER(QueryStats)), ("no_graph", _c_i32),
                ("subtract", _c_i32)]


class CSR(ctypes.Structure):
    _fields_ = [("n_queries", _c_i64), ("offsets", _c_p), ("ids", _c_p),
                ("on_device", _c_i32), ("reserved", _c_i32)]


class AutotuneResult(ctypes.Structure):
    _fields_ = [("cutover", _c_i32), ("inflight", _c_i32), ("tile_n", _c_i32),
                ("best_ms", ctypes.c_float), ("ms_cutover", ctypes.c_float * 9),
                ("ms_cutover_sub", ctypes.c_float * 9),
                ("ms_inflight", ctypes.c_float * 8), ("ms_tile", ctypes.c_float * 4),
                ("subtract", _c_i32)]


SCHEDULES = {"auto": 0, "levels": 1, "drain": 2, "immediate": 3}


class ServerOpts(ctypes.Structure):
    _fields_ = [("stream", _c_p), ("dtype", _c_i32), ("cutover", _c_i32),
                ("max_group", _c_i64), ("scratch_bytes", _c_i64), ("queue_capacity", _c_i64),
                ("schedule", _c_i32), ("reserved", _c_i32)]


class ServerStats(ctypes.Structure):
    _fields_ = [(k, _c_i64) for k in ("submitted", "admitted", "completed", "pending",
                                      "inserted", "steps", "launches", "retries", "rechecks",
                                      "refines", "gathered_tests", "dense_tests", "cutover",
                                      "max_group", "schedule")] + [("busy_seconds", _c_f64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TreeInfo(ctypes.Structure):
    _fields_ = [("n_items", _c_i64), ("capacity", _c_i64), ("d", _c_i32), ("row_width", _c_i32),
                ("levels", _c_i32), ("pooling", _c_i32), ("layout", _c_i32),
                ("prefix_level", _c_i32), ("formats", _c_u32), ("device", _c_i32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class GTError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None
ENTRY_POINTS = ("gt_build", "gt_insert", "gt_query", "gt_query_into", "gt_exhaustive",
                "gt_exhaustive_tree", "gt_read_rows",
                "gt_dense_scores", "gt_pair_bounds", "gt_query_static", "gt_server_create", "gt_server_submit",
                "gt_server_insert", "gt_server_step", "gt_server_poll", "gt_server_get_stats",
                "gt_server_free", "gt_autotune", "gt_set_tuning", "gt_set_wait_expiry",
                "gt_set_sm_limit", "gt_info", "gt_save", "gt_load",
                "gt_size", "gt_dim", "gt_levels", "gt_free", "gt_csr_free", "gt_last_error")


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libgt.so (building it first if asked); raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library missing: {_build.LIB} (run the build)")
        _build.build()
    lib = ctypes.CDLL(_build.LIB)
    P = _c_p
    lib.gt_build.argtypes = [P, _c_i64, _c_i32, ctypes.POINTER(BuildOpts), ctypes.POINTER(P)]
    lib.gt_insert.argtypes = [P, P, _c_i64, P]
    lib.gt_query.argtypes = [P, P, _c_i64, P, ctypes.POINTER(QueryOpts), ctypes.POINTER(CSR)]
    lib.gt_exhaustive_tree.argtypes = lib.gt_query.argtypes
    lib.gt_exhaustive.argtypes = [P, _c_i64, _c_i32, P, _c_i64, P, ctypes.POINTER(QueryOpts),
                                  ctypes.POINTER(CSR)]
    lib.gt_query_into.argtypes = [P, P, _c_i64, P, ctypes.POINTER(QueryOpts), P, P, _c_i64,
                                  ctypes.POINTER(_c_i64)]
    lib.gt_query_into.restype = _c_i32
    lib.gt_read_rows.argtypes = [P, _c_i32, _c_i32, _c_i64, _c_i64, P, P]
    lib.gt_dense_scores.argtypes = [P, P, _c_i64, _c_i32, P, P]
    lib.gt_pair_bounds.argtypes = [P, _c_i32, _c_i32, P, _c_i64, P, _c_i64, P, P]
    lib.gt_query_static.argtypes = [P, P, _c_i64, P, _c_i32, P, P, _c_i64,
                                    ctypes.POINTER(_c_i64), P]
    lib.gt_query_static.restype = _c_i32
    lib.gt_server_create.argtypes = [P, ctypes.POINTER(ServerOpts), ctypes.POINTER(P)]
    lib.gt_server_submit.argtypes = [P, P, P, P, _c_i64]
    lib.gt_server_insert.argtypes = [P, P, _c_i64]
    lib.gt_server_step.argtypes = [P, ctypes.POINTER(_c_i64)]
    lib.gt_server_poll.argtypes = [P, _c_i64, ctypes.POINTER(_c_i64), P, P, P, _c_i64, P]
    lib.gt_server_get_stats.argtypes = [P, ctypes.POINTER(ServerStats)]
    for f in ("gt_server_create", "gt_server_submit", "gt_server_insert", "gt_server_step",
              "gt_server_poll", "gt_server_get_stats"):
        getattr(lib, f).restype = _c_i32
    lib.gt_autotune.argtypes = [P, P, _c_i64, P, _c_i32, P, ctypes.POINTER(AutotuneResult)]
    lib.gt_autotune.restype = _c_i32
    lib.gt_set_tuning.argtypes = [P, _c_i32, _c_i32, _c_i32, _c_i32]
    lib.gt_set_tuning.restype = _c_i32
    lib.gt_set_wait_expiry.argtypes = [P, _c_i32]
    lib.gt_set_wait_expiry.restype = _c_i32
    lib.gt_set_sm_limit.argtypes = [P, _c_i32]
    lib.gt_set_sm_limit.restype = _c_i32
    lib.gt_info.argtypes = [P, ctypes.POINTER(TreeInfo)]
    lib.gt_info.restype = _c_i32
    lib.gt_save.argtypes = [P, ctypes.c_char_p]
    lib.gt_save.restype = _c_i32
    lib.gt_load.argtypes = [ctypes.c_char_p, P, ctypes.POINTER(P)]
    lib.gt_load.restype = _c_i32
    lib.gt_server_free.argtypes = [P]
    lib.gt_server_free.restype = None
    for f in ("gt_build", "gt_insert", "gt_query", "gt_exhaustive", "gt_exhaustive_tree",
              "gt_read_rows",
              "gt_dense_scores", "gt_pair_bounds"):
        getattr(lib, f).restype = _c_i32
    lib.gt_size.argtypes = [P]
    lib.gt_size.restype = _c_i64
    lib.gt_dim.argtypes = [P]
    lib.gt_dim.restype = _c_i32
    lib.gt_levels.argtypes = [P]
    lib.gt_levels.restype = _c_i32
    lib.gt_free.argtypes = [P]
    lib.gt_free.restype = None
    lib.gt_csr_free.argtypes = [ctypes.POINTER(CSR)]
    lib.gt_csr_free.restype = None
    lib.gt_last_error.argtypes = []
    lib.gt_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(st: int):
    if st != 0:
        raise GTError(st, load().gt_last_error().decode())


def _ptr(x, keep: list, dtype=np.float32):
    """Raw pointer of a numpy array or torch tensor (host or device)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):                       # torch tensor
        import torch
        want = {np.float32: torch.float32, np.int64: torch.int64}[dtype]
        if x.dtype != want or not x.is_contiguous():
            x = x.to(want).contiguous()
        keep.append(x)
        return ctypes.c_void_p(x.data_ptr())
    a = np.ascontiguousarray(x, dtype=dtype)
    keep.append(a)
    return ctypes.c_void_p(a.ctypes.data)


def _out_ptr(x, dtype):
    """Raw pointer of a caller-owned output buffer: a C-contiguous numpy array
    or torch tensor of exactly `dtype` (no copy is made, so nothing else will
    do)."""
    if hasattr(x, "data_ptr"):
        import torch
        want = {np.int64: torch.int64, np.int32: torch.int32}[dtype]
        if x.dtype != want or not x.is_contiguous():
            raise TypeError(f"output buffer must be a contiguous {want} tensor")
        return ctypes.c_void_p(x.data_ptr())
    if not isinstance(x, np.ndarray) or x.dtype != dtype or not x.flags.c_contiguous:
        raise TypeError(f"output buffer must be a C-contiguous {np.dtype(dtype)} array")
    return ctypes.c_void_p(x.ctypes.data)


def _static_arg(x, name: str, dtype: str, ndim: int = 1) -> int:
    """Check an argument of gt_query_static (a contiguous torch tensor of
    `dtype` with `ndim` dimensions) and return its length along dim 0."""
    if not hasattr(x, "data_ptr") or not hasattr(x, "is_cuda"):
        raise TypeError(f"{name} must be a torch tensor")
    if str(x.dtype) != f"torch.{dtype}":
        raise TypeError(f"{name} must be {dtype}, got {x.dtype}")
    if x.dim() != ndim:
        raise ValueError(f"{name} must have {ndim} dimension(s), got {x.dim()}")
    if not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return int(x.shape[0])


def exhaustive(F, Q, rho, max_batch: int = 0, scratch_bytes: int = 0,
               results_on_device: bool = False, stream=None, timing: bool = False) -> Result:
    """gt_exhaustive: {i : q.f_i >= rho} over the rows of F (N x d) for every
    query, by a dense scan of every (query, item) pair (no tree)."""
    lib = load()
    keep = []
    N, d = _rows(F)
    B = int(Q.shape[0])
    st = QueryStats()
    o = QueryOpts()
    o.stream = _stream_ptr(stream)
    o.dtype = GT_BF16
    o.max_batch = max_batch
    o.scratch_bytes = scratch_bytes
    o.results_on_device = 1 if results_on_device else 0
    o.timing = 1 if timing else 0
    o.stats = ctypes.pointer(st)
    if np.isscalar(rho):
        rho = np.full(B, rho, dtype=np.float32)
    csr = CSR()
    _check(lib.gt_exhaustive(_ptr(F, keep), N, d, _ptr(Q, keep), B, _ptr(rho, keep),
                             ctypes.byref(o), ctypes.byref(csr)))
    return Result(csr, st)


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _rows(x):
    return (int(x.shape[0]), int(x.shape[1]))


class Result:
    """Neighbour lists (CSR).  Host results are numpy arrays; device results
    stay library-owned until `free()` (raw device pointers)."""

    def __init__(self, csr: CSR, stats: QueryStats):
        self._csr = csr
        self.stats = stats.as_dict()
        self.on_device = bool(csr.on_device)
        B = csr.n_queries
        if not self.on_device:
            offs = np.ctypeslib.as_array((ctypes.c_int64 * (B + 1)).from_address(csr.offsets))
            self.offsets = offs.copy()
            n = int(self.offsets[-1])
            if n:
                self.ids = np.ctypeslib.as_array((ctypes.c_int32 * n).from_address(csr.ids)).copy()
            else:
                self.ids = np.zeros(0, dtype=np.int32)
            self.free()

    def neighbours(self, q: int) -> np.ndarray:
        return self.ids[self.offsets[q]:self.offsets[q + 1]]

    def free(self):
        if self._csr is not None:
            load().gt_csr_free(ctypes.byref(self._csr))
            self._csr = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Tree:
    """A pooled tree over a database F (N x d): gt_build / gt_insert / gt_query."""

    def __init__(self, F, perm=None, capacity: int = 0, formats=None, stream=None,
                 pooling: str = "sum", layout: str = "tree", prefix_level: int = 0):
        # formats None: the layout's default (tree: BF16 and FP8 rows; prefix:
        # BF16 prefix rows)
        lib = load()
        keep = []
        N, d = _rows(F)
        o = BuildOpts()
        o.stream = _stream_ptr(stream)
        o.perm = _ptr(perm, keep, np.int64) if perm is not None else None
        o.capacity = capacity
        o.formats = sum(1 << DTYPES[f] for f in formats) if formats is not None else 0
        o.pooling = POOLING[pooling] if isinstance(pooling, str) else int(pooling)
        o.layout = LAYOUTS[layout] if isinstance(layout, str) else int(layout)
        o.prefix_level = prefix_level
        self.layout = o.layout
        self.prefix_level = (prefix_level or 3) if o.layout == 1 else 0
        # stored rows: 2d entries ([max(f, 0), max(-f, 0)]) for signed descriptors
        self.row_width = 2 * d if o.pooling == POOLING["maxmin"] else d
        h = _c_p()
        _check(lib.gt_build(_ptr(F, keep), N, d, ctypes.byref(o), ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    @property
    def size(self) -> int:
        return int(load().gt_size(self._h))

    @property
    def dim(self) -> int:
        return int(load().gt_dim(self._h))

    @property
    def levels(self) -> int:
        return int(load().gt_levels(self._h))

    def insert(self, f, stream=None):
        keep = []
        n, _ = _rows(f)
        _check(load().gt_insert(self._h, _ptr(f, keep), n, _stream_ptr(stream)))

    def _search(self, fn, Q, rho, dtype, cutover, max_batch, scratch_bytes, results_on_device,
                stream, timing=False, graph=True, subtract=0):
        keep = []
        B = int(Q.shape[0])
        st = QueryStats()
        o = QueryOpts()
        o.stream = _stream_ptr(stream)
        o.dtype = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        o.cutover = cutover
        o.max_batch = max_batch
        o.scratch_bytes = scratch_bytes
        o.results_on_device = 1 if results_on_device else 0
        o.timing = 1 if timing else 0
        o.no_graph = 0 if graph else 1
        o.subtract = int(subtract)
        o.stats = ctypes.pointer(st)
        if np.isscalar(rho):
            rho = np.full(B, rho, dtype=np.float32)
        csr = CSR()
        _check(fn(self._h, _ptr(Q, keep), B, _ptr(rho, keep), ctypes.byref(o), ctypes.byref(csr)))
        return Result(csr, st)

    def query(self, Q, rho, dtype="bf16", cutover: int = -1, max_batch: int = 0,
              scratch_bytes: int = 0, results_on_device: bool = False, stream=None,
              timing: bool = False, graph: bool = True, subtract: int = 0) -> Result:
        """gt_query: {i : q.f_i >= rho} for every query (exact)."""
        return self._search(load().gt_query, Q, rho, dtype, cutover, max_batch, scratch_bytes,
                            results_on_device, stream, timing, graph, subtract)

    def query_into(self, Q, rho, offsets, ids, dtype="bf16", cutover: int = -1, stream=None,
                   subtract: int = 0) -> int:
        """gt_query_into: the sets of gt_query written into caller-owned CSR
        buffers `offsets` (B + 1 int64) and `ids` (int32), each a numpy array
        (ideally page-locked, e.g. a pinned torch tensor's numpy view) or a CUDA
        tensor.  Returns the number of neighbours written."""
        keep = []
        B = int(Q.shape[0])
        if np.isscalar(rho):
            rho = np.full(B, rho, dtype=np.float32)
        o = QueryOpts()
        o.stream = _stream_ptr(stream)
        o.dtype = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        o.cutover = cutover
        o.subtract = int(subtract)
        n = _c_i64(0)
        _check(load().gt_query_into(self._h, _ptr(Q, keep), B, _ptr(rho, keep), ctypes.byref(o),
                                    _out_ptr(offsets, np.int64), _out_ptr(ids, np.int32),
                                    int(ids.shape[0]), ctypes.byref(n)))
        return int(n.value)

    def exhaustive(self, Q, rho, max_batch: int = 0, scratch_bytes: int = 0,
                   results_on_device: bool = False, stream=None, timing: bool = False) -> Result:
        """gt_exhaustive_tree: the same sets by a dense scan of the tree's items."""
        return self._search(load().gt_exhaustive_tree, Q, rho, "bf16", 0, max_batch,
                            scratch_bytes, results_on_device, stream, timing)

    def query_static(self, Q, rho, offsets, ids, dtype="bf16", stream=None) -> int:
        """gt_query_static: the allocation-free query.  Q (B x d float32),
        rho (B float32), offsets (B+1 int64) and ids (int32) are contiguous
        CUDA tensors the caller owns; returns the number of neighbours
        written.  Arguments of the wrong type, shape or device are refused
        here, before the library is called (it reads and writes them in
        place, so a short or mistyped buffer would be accessed out of
        bounds)."""
        B = _static_arg(Q, "Q", "float32", ndim=2)
        if B < 1 or int(Q.shape[1]) != self.dim:
            raise ValueError(f"Q must have shape (B >= 1, {self.dim}), got {tuple(Q.shape)}")
        if _static_arg(rho, "rho", "float32") < B:
            raise ValueError(f"rho holds fewer than B = {B} thresholds")
        if _static_arg(offsets, "offsets", "int64") < B + 1:
            raise ValueError(f"offsets holds fewer than B + 1 = {B + 1} entries")
        n_ids = _static_arg(ids, "ids", "int32")
        for x in (Q, rho, offsets, ids):
            if not x.is_cuda:
                raise TypeError("gt_query_static takes CUDA tensors only")
        n = _c_i64(0)
        st = load().gt_query_static(
            self._h, ctypes.c_void_p(Q.data_ptr()), B,
            ctypes.c_void_p(rho.data_ptr()), DTYPES[dtype] if isinstance(dtype, str) else dtype,
            _out_ptr(offsets, np.int64), _out_ptr(ids, np.int32),
            n_ids, ctypes.byref(n), _stream_ptr(stream))
        if st != 0:
            err = GTError(st, load().gt_last_error().decode())
            err.n_results = n.value
            raise err
        return n.value

    def autotune(self, Q, rho, dtype="bf16", stream=None) -> dict:
        """gt_autotune: choose the cutover level and tests in flight per warp."""
        keep = []
        B = int(Q.shape[0])
        if np.isscalar(rho):
            rho = np.full(B, rho, dtype=np.float32)
        r = AutotuneResult()
        _check(load().gt_autotune(self._h, _ptr(Q, keep), B, _ptr(rho, keep),
                                  DTYPES[dtype] if isinstance(dtype, str) else dtype,
                                  _stream_ptr(stream), ctypes.byref(r)))
        ms = {f"cutover{c}": float(r.ms_cutover[c]) for c in range(1, 9) if r.ms_cutover[c] > 0}
        ms.update({f"cutover{c}_sub": float(r.ms_cutover_sub[c]) for c in range(2, 9)
                   if r.ms_cutover_sub[c] > 0})
        ms.update({f"inflight{g}": float(r.ms_inflight[i])
                   for i, g in enumerate((1, 2, 4, 9, 10, 12, 16, 32)) if r.ms_inflight[i] > 0})
        ms.update({f"tile{n}": float(r.ms_tile[i]) for i, n in enumerate((128, 256, 512, 1024))
                   if r.ms_tile[i] > 0})
        return {"cutover": r.cutover, "inflight": r.inflight, "tile_n": r.tile_n,
                "subtract": r.subtract, "best_ms": float(r.best_ms), "ms": ms}

    def set_tuning(self, dtype="bf16", cutover: int = -1, inflight: int = -1, tile: int = -1):
        """gt_set_tuning: pin the cutover level, tests in flight, GEMM tile."""
        _check(load().gt_set_tuning(self._h, DTYPES[dtype] if isinstance(dtype, str) else dtype,
                                    cutover, inflight, tile))

    def info(self) -> dict:
        """gt_info: sizes, row formats, pooling and layout of the tree."""
        r = TreeInfo()
        _check(load().gt_info(self._h, ctypes.byref(r)))
        return r.as_dict()

    def save(self, path: str):
        """gt_save: write a checkpoint gt_load rebuilds the same tree from."""
        _check(load().gt_save(self._h, os.fsencode(path)))

    @classmethod
    def load(cls, path: str, stream=None) -> "Tree":
        """gt_load: rebuild a tree from a checkpoint written by save()."""
        h = _c_p()
        _check(load().gt_load(os.fsencode(path), _stream_ptr(stream), ctypes.byref(h)))
        t = object.__new__(cls)
        t._h = h
        info = t.info()
        t.layout = info["layout"]
        t.prefix_level = info["prefix_level"]
        t.row_width = info["row_width"]
        return t

    def set_sm_limit(self, n: int):
        """gt_set_sm_limit: size later calls' grids for at most n SMs (0: all),
        so that calls on several trees and streams share the GPU."""
        _check(load().gt_set_sm_limit(self._h, int(n)))

    def set_wait_expiry(self, on: bool):
        """gt_set_wait_expiry: make the gather kernels' first bounded wait run
        out at once (the timeout path, for tests)."""
        _check(load().gt_set_wait_expiry(self._h, 1 if on else 0))

    def dense_scores(self, Q, level: int, stream=None) -> np.ndarray:
        """gt_dense_scores: raw tensor-core scores (B x rows of `level`)."""
        keep = []
        B = int(Q.shape[0])
        rows = (self.size + (1 << level) - 1) >> level
        out = np.empty((B, rows), dtype=np.float32)
        _check(load().gt_dense_scores(self._h, _ptr(Q, keep), B, level,
                                      ctypes.c_void_p(out.ctypes.data), _stream_ptr(stream)))
        return out

    def pair_bounds(self, level: int, dtype, Q, pairs, stream=None) -> np.ndarray:
        """gt_pair_bounds: the traversal's test of (query, pool) pairs at
        `level` in format `dtype`: an (n, 3) array of score, upper bound U and
        lower bound L per pair."""
        keep = []
        B = int(Q.shape[0])
        pr = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
        out = np.empty((pr.shape[0], 3), dtype=np.float32)
        _check(load().gt_pair_bounds(self._h, level, DTYPES[dtype] if isinstance(dtype, str) else dtype,
                                     _ptr(Q, keep), B, ctypes.c_void_p(pr.ctypes.data), pr.shape[0],
                                     ctypes.c_void_p(out.ctypes.data), _stream_ptr(stream)))
        return out

    def read_rows(self, level: int, dtype="f32", first: int = 0, count: int | None = None):
        fmt = DTYPES[dtype]
        N, d = self.size, self.row_width
        # level -1: a prefix-layout tree's prefix rows (one per item)
        rows = N if level < 0 else (N + (1 << level) - 1) >> level
        count = rows - first if count is None else count
        dt = {GT_F32: np.float32, GT_BF16: np.uint16, GT_FP8: np.uint8}[fmt]
        out = np.empty((count, d), dtype=dt)
        sc = np.empty(count, dtype=np.float32) if fmt == GT_FP8 else None
        _check(load().gt_read_rows(self._h, level, fmt, first, count,
                                   ctypes.c_void_p(out.ctypes.data),
                                   ctypes.c_void_p(sc.ctypes.data) if sc is not None else None))
        return (out, sc) if fmt == GT_FP8 else out

    def close(self):
        if getattr(self, "_h", None):
            load().gt_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop over a Tree (gt_server_*).

    submit() queues queries, insert() queues database rows, step() runs one
    engine iteration, poll() returns completed queries as
    (tag, ids, n_snapshot) tuples."""

    def __init__(self, tree: Tree, dtype="bf16", cutover: int = -1, max_group: int = 0,
                 scratch_bytes: int = 0, queue_capacity: int = 0, stream=None,
                 schedule: str = "auto"):
        o = ServerOpts()
        o.schedule = SCHEDULES[schedule] if isinstance(schedule, str) else int(schedule)
        o.stream = _stream_ptr(stream)
        o.dtype = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        o.cutover = cutover
        o.max_group = max_group
        o.scratch_bytes = scratch_bytes
        o.queue_capacity = queue_capacity
        h = _c_p()
        _check(load().gt_server_create(tree.handle, ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self.tree = tree
        self.d = tree.dim

    def submit(self, Q, rho, tags):
        keep = []
        Q = np.ascontiguousarray(Q, dtype=np.float32)
        n = int(Q.shape[0])
        rho = np.ascontiguousarray(np.broadcast_to(np.asarray(rho, np.float32), (n,)))
        tags = np.ascontiguousarray(np.asarray(tags, dtype=np.int64))
        _check(load().gt_server_submit(self._h, _ptr(Q, keep), _ptr(rho, keep),
                                       _ptr(tags, keep, np.int64), n))

    def insert(self, f):
        keep = []
        f = np.ascontiguousarray(f, dtype=np.float32)
        _check(load().gt_server_insert(self._h, _ptr(f, keep), int(f.shape[0])))

    def step(self) -> int:
        n = _c_i64(0)
        _check(load().gt_server_step(self._h, ctypes.byref(n)))
        return n.value

    def poll_arrays(self, max_queries: int = 65536, ids_cap: int = 1 << 22):
        """Completed queries as arrays: tags, offsets (CSR into ids), ids,
        tree-size snapshots."""
        if getattr(self, "_pbuf", None) is None or self._pbuf[0].size < max_queries:
            self._pbuf = (np.empty(max_queries, dtype=np.int64),
                          np.empty(max_queries + 1, dtype=np.int64),
                          np.empty(ids_cap, dtype=np.int32),
                          np.empty(max_queries, dtype=np.int64))
        tags, offs, ids, snap = self._pbuf
        n = _c_i64(0)
        _check(load().gt_server_poll(self._h, max_queries, ctypes.byref(n),
                                     ctypes.c_void_p(tags.ctypes.data),
                                     ctypes.c_void_p(offs.ctypes.data),
                                     ctypes.c_void_p(ids.ctypes.data), ids.size,
                                     ctypes.c_void_p(snap.ctypes.data)))
        k = n.value
        return tags[:k].copy(), offs[:k + 1].copy(), ids[:offs[k]].copy(), snap[:k].copy()

    def poll(self, max_queries: int = 65536, ids_cap: int = 1 << 22):
        """Completed queries as (tag, ids, n_snapshot) tuples."""
        tags, offs, ids, snap = self.poll_arrays(max_queries, ids_cap)
        return [(int(tags[k]), ids[offs[k]:offs[k + 1]], int(snap[k]))
                for k in range(tags.size)]

    def stats(self) -> dict:
        st = ServerStats()
        _check(load().gt_server_get_stats(self._h, ctypes.byref(st)))
        return st.as_dict()

    def close(self):
        if getattr(self, "_h", None):
            load().gt_server_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
