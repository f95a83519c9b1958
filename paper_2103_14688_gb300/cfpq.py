"""Thin Python binding of libcfpq (include/cfpq.h).

Argument marshalling only: every step of index creation runs inside the CUDA
library.  The functions keep the C names; the :class:`Context` wrapper adds
ownership and numpy conversion.  PyTorch supplies device memory (through the
allocator callbacks of ``cfpq_options``) and the CUDA stream.

The library must exist: :func:`load` builds it with nvcc for sm_103a when it
is missing and raises when that fails.  There is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from ctypes import (CFUNCTYPE, POINTER, Structure, c_char_p, c_double, c_int, c_int32, c_size_t,
                    c_uint8, c_uint32, c_uint64, c_void_p)
from typing import List, Optional, Sequence, Tuple

import numpy as np

CFPQ_OK = 0
CFPQ_ERR_INVALID_ARG = -1
CFPQ_ERR_OUT_OF_MEMORY = -2
CFPQ_ERR_BUFFER_TOO_SMALL = -3
CFPQ_ERR_TIMEOUT = -4
CFPQ_ERR_NOT_READY = -5
CFPQ_ERR_CUDA = -6
CFPQ_ERR_STATE = -7
CFPQ_ERR_UNSUPPORTED = -8

CFPQ_CLOSURE_AUTO = 0
CFPQ_CLOSURE_BITPACKED = 1
CFPQ_CLOSURE_TC_FP8 = 2
CFPQ_CLOSURE_TC_I8 = 3
CFPQ_CLOSURE_TC_FP4 = 4
CFPQ_TILES_DEFAULT = 0
CFPQ_TILES_FP8 = 1
CFPQ_TILES_FP4 = 2
CFPQ_TILES_FP8_128 = 3
CFPQ_TILES_NVFP4 = 4
CFPQ_LOOP_DEVICE = 0
CFPQ_LOOP_HOST = 1

cfpq_alloc_fn = CFUNCTYPE(c_void_p, c_size_t, c_void_p, c_void_p)
cfpq_free_fn = CFUNCTYPE(None, c_void_p, c_size_t, c_void_p, c_void_p)


class cfpq_options(Structure):
    _fields_ = [("struct_size", c_uint32), ("device", c_int32), ("max_iterations", c_uint32),
                ("max_rounds", c_uint32), ("closure_mode", c_uint32), ("loop_mode", c_uint32),
                ("profile", c_uint32), ("no_single_cta", c_uint32), ("gather_slices", c_uint32),
                ("memory_budget", c_size_t), ("alloc", cfpq_alloc_fn), ("free", cfpq_free_fn),
                ("alloc_user", c_void_p), ("tile_format", c_uint32), ("no_autotune", c_uint32),
                ("tile_ratio", c_uint32)]


class cfpq_rsm(Structure):
    _fields_ = [("n_states", c_uint32), ("n_boxes", c_uint32), ("start_box", c_uint32), ("n_trans", c_uint32),
                ("box_start", POINTER(c_uint32)), ("state_box", POINTER(c_uint32)),
                ("state_final", POINTER(c_uint8)), ("tr_from", POINTER(c_uint32)),
                ("tr_kind", POINTER(c_uint32)), ("tr_sym", POINTER(c_uint32)), ("tr_to", POINTER(c_uint32))]


class cfpq_run_stats(Structure):
    _fields_ = [("iterations", c_uint32), ("rounds", c_uint32), ("status", c_uint32), ("gpu_launches", c_uint32),
                ("edges_added", c_uint64), ("closure_bits", c_uint64), ("m3_bits", c_uint64),
                ("row_ors", c_uint64), ("rows_changed", c_uint64), ("row_bytes", c_uint64),
                ("tile_mmas", c_uint64), ("closure_blocks", c_uint64),
                ("device_bytes", c_uint64), ("ms_total", c_double), ("ms_closure", c_double),
                ("ms_setup", c_double), ("ms_loop", c_double),
                ("closure_launches", c_uint32), ("pad_", c_uint32),
                ("tile_kstages", c_uint64), ("ms_gather", c_double), ("ms_tile_operands", c_double),
                ("ms_tile_products", c_double), ("gather_launches", c_uint32), ("tile_launches", c_uint32),
                ("tile_operand_bytes", c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class cfpq_tuning(Structure):
    _fields_ = [("struct_size", c_uint32), ("tuned", c_uint32), ("tile_format", c_uint32), ("edge_ratio", c_uint32),
                ("edge_ratio_hbm", c_uint32), ("edge_ratio_formula", c_uint32), ("probe_status", c_int32),
                ("gather_gbs", c_double),
                ("gather_gbs_hbm", c_double), ("read_l2_gbs", c_double), ("read_hbm_gbs", c_double),
                ("fp8_tflops", c_double), ("fp4_tflops", c_double), ("fp8_128_tflops", c_double),
                ("nvfp4_tflops", c_double), ("probe_ms", c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "struct_size"}


class cfpq_query(Structure):
    _fields_ = [("n_vertices", c_uint32), ("n_terminals", c_uint32), ("n_edges", c_size_t),
                ("src", POINTER(c_uint32)), ("label", POINTER(c_uint32)), ("dst", POINTER(c_uint32)),
                ("rsm", POINTER(cfpq_rsm))]


_lock = threading.Lock()
_lib = None


class CfpqError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def library_path() -> str:
    from . import build as _b
    return _b.LIB


def load():
    """Load libcfpq.so, building it first if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _b
        path = _b.build()
        lib = ctypes.CDLL(path)
        _declare(lib)
        _lib = lib
        return lib


def _declare(lib):
    P = c_void_p
    u32p = POINTER(c_uint32)
    u64p = POINTER(c_uint64)
    sig = {
        "cfpq_default_options": (c_int, [POINTER(cfpq_options)]),
        "cfpq_create": (c_int, [POINTER(P), POINTER(cfpq_options), P]),
        "cfpq_destroy": (c_int, [P]),
        "cfpq_load_graph": (c_int, [P, c_uint32, c_uint32, c_size_t, u32p, u32p, u32p]),
        "cfpq_load_graph_device": (c_int, [P, c_uint32, c_uint32, c_size_t, P, P, P]),
        "cfpq_load_graph_device_noalloc": (c_int, [P, c_uint32, c_uint32, c_size_t, P, P, P]),
        "cfpq_load_rsm": (c_int, [P, POINTER(cfpq_rsm)]),
        "cfpq_shard_begin": (c_int, [P, c_uint32, c_uint32]),
        "cfpq_shard_step": (c_int, [P, P, POINTER(c_uint64)]),
        "cfpq_shard_apply": (c_int, [P, P, POINTER(c_int)]),
        "cfpq_shard_stats": (c_int, [P, POINTER(cfpq_run_stats)]),
        "cfpq_run": (c_int, [P, POINTER(cfpq_run_stats)]),
        "cfpq_run_sources": (c_int, [P, POINTER(c_uint32), c_uint32, POINTER(cfpq_run_stats)]),
        "cfpq_count_index": (c_int, [P, u64p, u64p]),
        "cfpq_tune": (c_int, [P, c_int, POINTER(cfpq_tuning)]),
        "cfpq_check_bounded_wait": (c_int, [P, c_uint64, POINTER(c_int)]),
        "cfpq_set_start": (c_int, [P, P, c_uint32, c_uint32]),
        "cfpq_get_reachable": (c_int, [P, c_uint32, u32p, u32p, c_size_t, POINTER(c_size_t)]),
        "cfpq_count_reachable": (c_int, [P, c_uint32, u64p]),
        "cfpq_get_reachable_bits": (c_int, [P, c_uint32, P]),
        "cfpq_get_closure_rows": (c_int, [P, c_uint32, u32p, u32p, P]),
        "cfpq_extract_paths": (c_int, [P, c_uint32, c_uint32, c_uint32, c_uint32, c_size_t, u32p, c_size_t,
                                       POINTER(c_size_t), POINTER(c_size_t), POINTER(c_int)]),
        "cfpq_batch_run": (c_int, [P, c_uint32, POINTER(cfpq_query), POINTER(cfpq_run_stats),
                                   POINTER(cfpq_run_stats)]),
        "cfpq_batch_get_reachable_bits": (c_int, [P, c_uint32, c_uint32, P]),
        "cfpq_server_create": (c_int, [POINTER(P), POINTER(cfpq_options), P, c_uint32, c_uint32, c_size_t,
                                       u32p, u32p, u32p]),
        "cfpq_server_destroy": (c_int, [P]),
        "cfpq_submit": (c_int, [P, POINTER(cfpq_rsm), u64p]),
        "cfpq_server_step": (c_int, [P, u32p, u32p]),
        "cfpq_poll": (c_int, [P, c_uint64, POINTER(c_int)]),
        "cfpq_result_reachable_bits": (c_int, [P, c_uint64, c_uint32, P]),
        "cfpq_release": (c_int, [P, c_uint64]),
        "cfpq_tc_bool_product": (c_int, [c_uint32, c_int, P, P, P, P]),
        "cfpq_status_string": (c_char_p, [c_int]),
        "cfpq_last_error": (c_char_p, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint32))


def _u32p(a: np.ndarray):
    return a.ctypes.data_as(POINTER(c_uint32))


class RSMArgs:
    """Holds a cfpq_rsm and the arrays it points to."""

    def __init__(self, r):
        self.box_start = _u32(r.box_start)
        self.state_box = _u32(r.state_box)
        self.state_final = np.ascontiguousarray(r.state_final, dtype=np.uint8)
        self.tr_from = _u32(r.tr_from)
        self.tr_kind = _u32(r.tr_kind)
        self.tr_sym = _u32(r.tr_sym)
        self.tr_to = _u32(r.tr_to)
        self.c = cfpq_rsm(r.n_states, r.n_boxes, r.start_box, len(self.tr_from), _u32p(self.box_start),
                          _u32p(self.state_box), self.state_final.ctypes.data_as(POINTER(c_uint8)),
                          _u32p(self.tr_from), _u32p(self.tr_kind), _u32p(self.tr_sym), _u32p(self.tr_to))


class _TorchAllocator:
    """Routes the library's device allocations to PyTorch's caching allocator."""

    def __init__(self, device: int):
        import torch
        self.torch = torch
        self.device = device

        def alloc(nbytes, stream, user):
            try:
                return self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, stream or 0)
            except Exception:
                return None

        def free(ptr, nbytes, stream, user):
            self.torch.cuda.caching_allocator_delete(ptr)

        self.alloc = cfpq_alloc_fn(alloc)
        self.free = cfpq_free_fn(free)


def default_options(**kw) -> cfpq_options:
    lib = load()
    o = cfpq_options()
    lib.cfpq_default_options(ctypes.byref(o))
    names = {f for f, _ in cfpq_options._fields_}
    for k, v in kw.items():
        # a ctypes structure would keep a misspelt name as a plain attribute
        if k not in names:
            raise TypeError(f"unknown cfpq option {k!r}")
        setattr(o, k, v)
    return o


def status_string(code: int) -> str:
    return load().cfpq_status_string(code).decode()


class Context:
    """A cfpq_ctx on one device and stream.

    ``use_torch`` routes allocations through torch's caching allocator and
    uses torch's current stream (the default); otherwise the library uses
    cudaMallocAsync on the legacy default stream.
    """

    def __init__(self, device: int = 0, use_torch: bool = True, stream=None, **options):
        self.lib = load()
        self._alloc = None
        o = default_options(device=device, **options)
        if use_torch:
            import torch
            torch.cuda.init()
            self._alloc = _TorchAllocator(device)
            o.alloc = self._alloc.alloc
            o.free = self._alloc.free
            if stream is None:
                with torch.cuda.device(device):
                    stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        self._opt = o
        h = c_void_p()
        self._check(self.lib.cfpq_create(ctypes.byref(h), ctypes.byref(o), c_void_p(stream or 0)), "cfpq_create",
                    with_ctx=False)
        self.h = h
        self.n = None
        self.n_boxes = None
        self.n_states = None

    # -- plumbing --
    def _check(self, rc: int, what: str, with_ctx: bool = True):
        if rc != CFPQ_OK:
            msg = self.lib.cfpq_status_string(rc).decode()
            if with_ctx and getattr(self, "h", None):
                detail = self.lib.cfpq_last_error(self.h)
                if detail:
                    msg += ": " + detail.decode()
            raise CfpqError(rc, f"{what}: {msg}")

    def close(self):
        if getattr(self, "h", None):
            self.lib.cfpq_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- inputs --
    def load_graph(self, g):
        s, l, d = _u32(g.src), _u32(g.lbl), _u32(g.dst)
        self._check(self.lib.cfpq_load_graph(self.h, g.n, g.n_terminals, len(s), _u32p(s), _u32p(l), _u32p(d)),
                    "cfpq_load_graph")
        self.n = g.n

    def load_graph_device(self, n: int, n_terminals: int, src, lbl, dst):
        """src/lbl/dst: torch CUDA tensors of int32/uint32 (same length)."""
        m = int(src.numel())
        self._check(self.lib.cfpq_load_graph_device(self.h, n, n_terminals, m, c_void_p(src.data_ptr()),
                                                    c_void_p(lbl.data_ptr()), c_void_p(dst.data_ptr())),
                    "cfpq_load_graph_device")
        self.n = n

    def load_rsm(self, r):
        self._rsm = RSMArgs(r)
        self._check(self.lib.cfpq_load_rsm(self.h, ctypes.byref(self._rsm.c)), "cfpq_load_rsm")
        self.n_boxes = r.n_boxes
        self.n_states = r.n_states

    # -- index creation --
    def run(self) -> cfpq_run_stats:
        st = cfpq_run_stats()
        self._check(self.lib.cfpq_run(self.h, ctypes.byref(st)), "cfpq_run")
        return st

    def run_sources(self, sources) -> cfpq_run_stats:
        """Index creation for the source vertices only (exact rows for them)."""
        src = _u32(np.asarray(sources, dtype=np.uint32).reshape(-1))
        st = cfpq_run_stats()
        self._check(self.lib.cfpq_run_sources(self.h, _u32p(src) if len(src) else None, len(src), ctypes.byref(st)),
                    "cfpq_run_sources")
        return st

    def set_start(self, words=None):
        """Start the next runs from the given M2 per box (uint64 words
        [n_boxes, n, ceil(n/64)], as reachable_words returns them per box);
        None clears the start."""
        if words is None:
            self._check(self.lib.cfpq_set_start(self.h, None, 0, 0), "cfpq_set_start")
            return
        w = np.ascontiguousarray(np.asarray(words, dtype=np.uint64))
        if w.ndim != 3:
            raise ValueError("start words must be [n_boxes, n, ceil(n/64)]")
        self._check(self.lib.cfpq_set_start(self.h, c_void_p(w.ctypes.data), w.shape[0], w.shape[1]),
                    "cfpq_set_start")

    def check_bounded_wait(self, limit_ns: int) -> bool:
        """Run the kernels' bounded mbarrier wait on a barrier nothing
        arrives at; True when it gave up after ``limit_ns``."""
        t = c_int()
        self._check(self.lib.cfpq_check_bounded_wait(self.h, c_uint64(limit_ns), ctypes.byref(t)),
                    "cfpq_check_bounded_wait")
        return bool(t.value)

    def tune(self, force: bool = False) -> cfpq_tuning:
        """The autotuner's measurements and choices for this context's device
        (runs its probe query once per device and process, or again with
        force)."""
        t = cfpq_tuning()
        t.struct_size = ctypes.sizeof(cfpq_tuning)
        self._check(self.lib.cfpq_tune(self.h, 1 if force else 0, ctypes.byref(t)), "cfpq_tune")
        return t

    def count_index(self) -> Tuple[int, int]:
        a, b = c_uint64(), c_uint64()
        self._check(self.lib.cfpq_count_index(self.h, ctypes.byref(a), ctypes.byref(b)), "cfpq_count_index")
        return a.value, b.value

    # -- results --
    def reachable_words(self, box: int = 0) -> np.ndarray:
        wn = (self.n + 63) // 64
        out = np.zeros(self.n * wn, dtype=np.uint64)
        self._check(self.lib.cfpq_get_reachable_bits(self.h, box, c_void_p(out.ctypes.data)),
                    "cfpq_get_reachable_bits")
        return out.reshape(self.n, wn)

    def reachable_bits(self, box: int = 0) -> np.ndarray:
        w = self.reachable_words(box)
        return np.unpackbits(w.view(np.uint8), axis=1, bitorder="little")[:, : self.n].astype(bool)

    def reachable_pairs(self, box: int = 0) -> np.ndarray:
        cnt = c_size_t()
        rc = self.lib.cfpq_get_reachable(self.h, box, None, None, 0, ctypes.byref(cnt))
        self._check(rc, "cfpq_get_reachable")
        k = cnt.value
        s = np.zeros(max(k, 1), dtype=np.uint32)
        d = np.zeros(max(k, 1), dtype=np.uint32)
        self._check(self.lib.cfpq_get_reachable(self.h, box, _u32p(s), _u32p(d), k, ctypes.byref(cnt)),
                    "cfpq_get_reachable")
        return np.stack([s[:k], d[:k]], axis=1)

    def count_reachable(self, box: int = 0) -> int:
        c = c_uint64()
        self._check(self.lib.cfpq_count_reachable(self.h, box, ctypes.byref(c)), "cfpq_count_reachable")
        return c.value

    def closure_rows(self, rows: Sequence[Tuple[int, int]]) -> np.ndarray:
        """Rows of C3 as bool [len(rows), Q*n], column t*n + y."""
        rs = _u32([a for a, _ in rows])
        rv = _u32([b for _, b in rows])
        N = self.n_states * self.n
        wN = (N + 63) // 64
        out = np.zeros(len(rows) * wN, dtype=np.uint64)
        self._check(self.lib.cfpq_get_closure_rows(self.h, len(rows), _u32p(rs), _u32p(rv),
                                                   c_void_p(out.ctypes.data)), "cfpq_get_closure_rows")
        return np.unpackbits(out.reshape(len(rows), wN).view(np.uint8), axis=1, bitorder="little")[:, :N].astype(bool)

    def extract_paths(self, box: int, vs: int, vf: int, max_len: int, max_paths: int = 1 << 16,
                      edge_cap: int = 1 << 22):
        edges = np.zeros(3 * max(edge_cap, 1), dtype=np.uint32)
        offs = (c_size_t * (max_paths + 1))()
        npaths = c_size_t()
        trunc = c_int()
        self._check(self.lib.cfpq_extract_paths(self.h, box, vs, vf, max_len, max_paths, _u32p(edges), edge_cap,
                                                offs, ctypes.byref(npaths), ctypes.byref(trunc)),
                    "cfpq_extract_paths")
        out = []
        for i in range(npaths.value):
            a, b = offs[i], offs[i + 1]
            out.append(tuple((int(edges[3 * j]), int(edges[3 * j + 1]), int(edges[3 * j + 2])) for j in range(a, b)))
        return out, bool(trunc.value)

    # -- batches --
    def batch_run(self, queries) -> Tuple[List[cfpq_run_stats], cfpq_run_stats]:
        keep = []
        arr = (cfpq_query * len(queries))()
        for i, (g, r) in enumerate(queries):
            s, l, d = _u32(g.src), _u32(g.lbl), _u32(g.dst)
            ra = RSMArgs(r)
            keep.append((s, l, d, ra))
            arr[i] = cfpq_query(g.n, g.n_terminals, len(s), _u32p(s), _u32p(l), _u32p(d), ctypes.pointer(ra.c))
        per = (cfpq_run_stats * len(queries))()
        tot = cfpq_run_stats()
        self._check(self.lib.cfpq_batch_run(self.h, len(queries), arr, per, ctypes.byref(tot)), "cfpq_batch_run")
        self._batch_n = [g.n for g, _ in queries]
        return list(per), tot

    def batch_reachable_words(self, q: int, box: int = 0) -> np.ndarray:
        """M2^box of query q of the last batch as bit rows, uint64 [n, ceil(n/64)]."""
        n = self._batch_n[q]
        wn = (n + 63) // 64
        out = np.zeros(n * wn, dtype=np.uint64)
        self._check(self.lib.cfpq_batch_get_reachable_bits(self.h, q, box, c_void_p(out.ctypes.data)),
                    "cfpq_batch_get_reachable_bits")
        return out.reshape(n, wn)

    def batch_reachable_bits(self, q: int, box: int = 0) -> np.ndarray:
        n = self._batch_n[q]
        w = self.batch_reachable_words(q, box)
        return np.unpackbits(w.view(np.uint8), axis=1, bitorder="little")[:, :n].astype(bool)


class Server:
    """A cfpq_server: resident graph, continuously batched RSM queries."""

    def __init__(self, g, device: int = 0, use_torch: bool = True, stream=None, **options):
        self.lib = load()
        self._alloc = None
        o = default_options(device=device, **options)
        if use_torch:
            import torch
            torch.cuda.init()
            self._alloc = _TorchAllocator(device)
            o.alloc = self._alloc.alloc
            o.free = self._alloc.free
            if stream is None:
                with torch.cuda.device(device):
                    stream = torch.cuda.current_stream().cuda_stream
            # without memory_budget the server admits queries into the device's
            # free memory at creation: return PyTorch's cached blocks first (an
            # earlier server's or context's buffers would otherwise count as used)
            if not o.memory_budget:
                with torch.cuda.device(device):
                    torch.cuda.synchronize()
                    torch.cuda.empty_cache()
        s, l, d = _u32(g.src), _u32(g.lbl), _u32(g.dst)
        h = c_void_p()
        rc = self.lib.cfpq_server_create(ctypes.byref(h), ctypes.byref(o), c_void_p(stream or 0), g.n, g.n_terminals,
                                         len(s), _u32p(s), _u32p(l), _u32p(d))
        if rc != CFPQ_OK:
            raise CfpqError(rc, "cfpq_server_create: " + status_string(rc))
        self.h = h
        self.n = g.n
        self._keep = {}

    def close(self):
        if getattr(self, "h", None):
            self.lib.cfpq_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, r) -> int:
        ra = RSMArgs(r)
        t = c_uint64()
        rc = self.lib.cfpq_submit(self.h, ctypes.byref(ra.c), ctypes.byref(t))
        if rc != CFPQ_OK:
            raise CfpqError(rc, "cfpq_submit: " + status_string(rc))
        self._keep[t.value] = (ra, r.n_boxes)
        return t.value

    def step(self) -> Tuple[int, int]:
        a, b = c_uint32(), c_uint32()
        rc = self.lib.cfpq_server_step(self.h, ctypes.byref(a), ctypes.byref(b))
        if rc != CFPQ_OK:
            raise CfpqError(rc, "cfpq_server_step: " + status_string(rc))
        return a.value, b.value

    def poll(self, ticket: int) -> bool:
        d = c_int()
        rc = self.lib.cfpq_poll(self.h, ticket, ctypes.byref(d))
        if rc != CFPQ_OK:
            raise CfpqError(rc, "cfpq_poll: " + status_string(rc))
        return bool(d.value)

    def result_words(self, ticket: int, box: int = 0) -> np.ndarray:
        """M2^box of a finished query as bit rows, uint64 [n, ceil(n/64)]."""
        wn = (self.n + 63) // 64
        out = np.zeros(self.n * wn, dtype=np.uint64)
        rc = self.lib.cfpq_result_reachable_bits(self.h, ticket, box, c_void_p(out.ctypes.data))
        if rc != CFPQ_OK:
            raise CfpqError(rc, "cfpq_result_reachable_bits: " + status_string(rc))
        return out.reshape(self.n, wn)

    def result_bits(self, ticket: int, box: int = 0) -> np.ndarray:
        w = self.result_words(ticket, box)
        return np.unpackbits(w.view(np.uint8), axis=1, bitorder="little")[:, : self.n].astype(bool)

    def release(self, ticket: int):
        rc = self.lib.cfpq_release(self.h, ticket)
        if rc != CFPQ_OK:
            raise CfpqError(rc, "cfpq_release: " + status_string(rc))
        self._keep.pop(ticket, None)


class ColumnShardEngine:
    """This rank's part of one query split by closure columns (the engine of
    ``shard.run_column_sharded``): a Context holding the whole graph and RSM,
    computing the closure on the columns it is given.  Slices and full rows
    are int64 torch tensors on the context's device ([B, n, words])."""

    def __init__(self, ctx: "Context", g, r):
        import torch
        self.ctx, self.lib = ctx, ctx.lib
        ctx.load_graph(g)
        ctx.load_rsm(r)
        self.n, self.B = g.n, r.n_boxes
        self.W = (g.n + 127) // 128 * 2
        self.device = torch.device("cuda", ctx._opt.device)
        self.slice = None

    def begin(self, col0: int, col1: int):
        import torch
        self.ctx._check(self.lib.cfpq_shard_begin(self.ctx.h, col0, col1), "cfpq_shard_begin")
        self.slice = torch.zeros((self.B, self.n, (col1 - col0) // 64), dtype=torch.int64, device=self.device)

    def step(self):
        k = c_uint64()
        self.ctx._check(self.lib.cfpq_shard_step(self.ctx.h, c_void_p(self.slice.data_ptr()), ctypes.byref(k)),
                        "cfpq_shard_step")
        self.last_new = k.value
        return self.slice

    def apply(self, full) -> bool:
        import torch
        full = full.to(self.device).contiguous()
        assert full.dtype == torch.int64 and tuple(full.shape) == (self.B, self.n, self.W)
        d = c_int()
        self.ctx._check(self.lib.cfpq_shard_apply(self.ctx.h, c_void_p(full.data_ptr()), ctypes.byref(d)),
                        "cfpq_shard_apply")
        return bool(d.value)

    def stats(self) -> cfpq_run_stats:
        st = cfpq_run_stats()
        self.ctx._check(self.lib.cfpq_shard_stats(self.ctx.h, ctypes.byref(st)), "cfpq_shard_stats")
        return st


def tc_bool_product(a: np.ndarray, b: np.ndarray, use_int8: bool = False, stream=None) -> np.ndarray:
    """Boolean product of two n x n bool matrices on the tensor cores."""
    lib = load()
    n = a.shape[0]
    wn = (n + 63) // 64

    def pack(m):
        pad = np.zeros((n, wn * 64), dtype=bool)
        pad[:, :n] = m
        return np.ascontiguousarray(np.packbits(pad, axis=1, bitorder="little").view(np.uint64))

    pa, pb = pack(a), pack(b)
    out = np.zeros((n, wn), dtype=np.uint64)
    rc = lib.cfpq_tc_bool_product(n, 1 if use_int8 else 0, c_void_p(pa.ctypes.data), c_void_p(pb.ctypes.data),
                                  c_void_p(out.ctypes.data), c_void_p(stream or 0))
    if rc != CFPQ_OK:
        raise CfpqError(rc, "cfpq_tc_bool_product: " + status_string(rc))
    return np.unpackbits(out.view(np.uint8), axis=1, bitorder="little")[:, :n].astype(bool)
