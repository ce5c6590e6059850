"""Python binding of libcox.so (the C ABI declared in include/cox.h).

Argument marshalling only: every step of every op runs in the library's CUDA
kernels.  ``cox_*`` functions mirror the C entry points one for one (plain
ints for pointers and the stream) and return the status code; the lower-case
helpers take torch CUDA tensors, allocate outputs with torch, pass
``data_ptr()`` and torch's current stream, and raise ``CoxError`` on a
non-OK status.  There is no fallback: if libcox.so is missing the import of
the library fails.
"""
from __future__ import annotations

import ctypes
import os

from .build import lib_path

# ------------------------------------------------------------------ codes
COX_OK, COX_EINVAL, COX_EUNSUPPORTED, COX_ECUDA, COX_ENOMEM, COX_ETIMEOUT, COX_EBUSY = range(7)
COX_I32, COX_U32, COX_F32, COX_U8 = 0, 1, 2, 3
COX_SUM, COX_MIN, COX_MAX, COX_AND, COX_OR, COX_XOR = range(6)
(COX_SHFL_IDX, COX_SHFL_UP, COX_SHFL_DOWN, COX_SHFL_XOR,
 COX_BALLOT, COX_ANY, COX_ALL, COX_MATCH_ANY) = range(8)
COX_SCOPE_TILE, COX_SCOPE_BLOCK, COX_SCOPE_GRID = 0, 1, 2
COX_GRID_SUB_MIN, COX_GRID_NORMALIZE = 0, 1
(COX_CG_SIZE, COX_CG_RANK, COX_CG_SHFL, COX_CG_SHFL_UP, COX_CG_SHFL_DOWN, COX_CG_BALLOT, COX_CG_ANY, COX_CG_ALL,
 COX_CG_REDUCE_SUM, COX_CG_SCAN_SUM) = range(10)
(COX_F_COMPENSATED, COX_F_FP64_COMBINE, COX_F_WS_READY, COX_F_NATIVE_MATCH, COX_F_DIRECT_ATOMICS,
 COX_F_BALLOT_MATCH) = 1, 2, 4, 8, 16, 32
FULL_MASK = 0xFFFFFFFF

_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_U = ctypes.c_uint
_SZ = ctypes.c_size_t

# name -> (restype, argtypes), in the order of include/cox.h
SIGNATURES = {
    "cox_status_string": (ctypes.c_char_p, [_I]),
    "cox_version": (_I, []),
    "cox_shfl": (_I, [_I, _I, _I, _I, _P, _P, _I64, _I, ctypes.c_uint32, _P]),
    "cox_tile_reduce": (_I, [_I, _I, _I, _I, _I, _P, _P, _I64, _U, _P, _P, _SZ, _P]),
    "cox_tile_reduce_workspace": (_SZ, [_I, _I64, _I]),
    "cox_tile_scan": (_I, [_I, _I, _I, _I, _P, _P, _I64, _U, _P]),
    "cox_scan": (_I, [_I, _I, _I, _I, _P, _P, _I64, _U, _I, _P, _SZ, _P]),
    "cox_scan_workspace": (_SZ, [_I, _I64]),
    "cox_grid_broadcast": (_I, [_I, _I, _P, _P, _I64, _P, _SZ, _P]),
    "cox_grid_broadcast_workspace": (_SZ, [_I64]),
    "cox_coalesced": (_I, [_I, _I, _I, _P, _P, _P, _I64, _I, _P]),
    "cox_filter_aggregated": (_I, [_I, _P, _I64, _I64, _P, _P, _P]),
    "cox_vote_stats": (_I, [_I, _I, _P, _I64, _I64, _P, _P]),
    "cox_integral_image": (_I, [_I, _I64, _I64, _I64, _P, _P, _P, _SZ, _P]),
    "cox_integral_image_workspace": (_SZ, [_I64, _I64, _I64]),
    "cox_ballot_compact": (_I, [_I, _I, _I, _P, _I64, _I64, _P, _P, _P, _SZ, _U, _P]),
    "cox_ballot_compact_workspace": (_SZ, [_I64, _I]),
    "cox_ballot_compact_static": (_I, [_I, _I, _I, _P, _I64, _I64, _P, _P, _P]),
    "cox_match_histogram": (_I, [_I, _I, _I, _P, _I64, _I, _P, _P, _U, _P]),
    "cox_batch_workspace": (_SZ, [_I64]),
    "cox_batch_prepare": (_I, [_I64, _P, _P, _SZ, _P]),
    "cox_batch_sum_hist": (_I, [_I64, _P, _P, _P, _P, _SZ, _P, _P, _P, _P]),
    "cox_batch_percall_scratch": (_SZ, [_I64]),
    "cox_batch_percall": (_I, [_I64, _P, _P, _P, _P, _P, _P, _SZ, _P, _P]),
    "cox_batch_graph_create": (_I, [_I64, _P, _P, _P, _P, _SZ, _P, _P, _P, _P]),
    "cox_graph_launch": (_I, [_P, _P]),
    "cox_graph_destroy": (None, [_P]),
    "cox_batch_autotune": (_I, [_I64, _P, _P, _P, _SZ, _P, _P, _I, ctypes.c_char_p, _P, _P, _P]),
    "cox_batch_tune_lookup": (_I, [ctypes.c_char_p, _I64, _I64, _P]),
    "cox_server_create": (_I, [_SZ, _I, _P]),
    "cox_server_submit": (_I, [_P, _P, _P]),
    "cox_server_submit_many": (_I, [_P, _P, _I64, _P]),
    "cox_server_poll": (_I, [_P, ctypes.c_uint64, _P]),
    "cox_server_wait": (_I, [_P, ctypes.c_uint64, ctypes.c_double]),
    "cox_server_result": (_I, [_P, ctypes.c_uint64, _P, _P]),
    "cox_server_release": (_I, [_P, ctypes.c_uint64]),
    "cox_server_get_stats": (_I, [_P, _P]),
    "cox_server_destroy": (None, [_P]),
    "cox_server_run_trace": (_I, [_P, _P, _I64, _P, _P]),
    "cox_percall_scratch": (_SZ, [_I64]),
    "cox_percall_run_trace": (_I, [_P, _I64, _P, _SZ, _P, _P]),
    "cox_device_status": (_I, [_P]),
    "cox_set_spin_limit": (None, [ctypes.c_uint32]),
}

_lib = None


class CoxError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = int(status)
        super().__init__(f"{what}: {status_string(status)}" if what else status_string(status))


def lib() -> ctypes.CDLL:
    """The loaded libcox.so (raises ImportError if it was never built)."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise ImportError(f"libcox.so is not built ({path}); run __graft_entry__.build()")
        handle = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(handle, name)
            f.restype = res
            f.argtypes = args
        _lib = handle
    return _lib


def status_string(s: int) -> str:
    return lib().cox_status_string(int(s)).decode()


# ------------------------------------------------------- raw C-ABI mirrors
def cox_version() -> int:
    return lib().cox_version()


def cox_shfl(fn, dt, width, block_dim, d_in, d_out, n, param, mask, stream) -> int:
    return lib().cox_shfl(fn, dt, width, block_dim, d_in, d_out, n, param, mask, stream)


def cox_tile_reduce(op, dt, width, block_dim, scope, d_in, d_out, n, flags, d_err, d_ws, ws_bytes, stream) -> int:
    return lib().cox_tile_reduce(op, dt, width, block_dim, scope, d_in, d_out, n, flags, d_err, d_ws, ws_bytes,
                                 stream)


def cox_tile_reduce_workspace(scope, n, block_dim) -> int:
    return lib().cox_tile_reduce_workspace(scope, n, block_dim)


def cox_tile_scan(op, dt, width, block_dim, d_in, d_out, n, flags, stream) -> int:
    return lib().cox_tile_scan(op, dt, width, block_dim, d_in, d_out, n, flags, stream)


def cox_scan(op, dt, scope, block_dim, d_in, d_out, n, flags, exclusive, d_ws, ws_bytes, stream) -> int:
    return lib().cox_scan(op, dt, scope, block_dim, d_in, d_out, n, flags, exclusive, d_ws, ws_bytes, stream)


def cox_scan_workspace(scope, n) -> int:
    return lib().cox_scan_workspace(scope, n)


def cox_grid_broadcast(op, dt, d_in, d_out, n, d_ws, ws_bytes, stream) -> int:
    return lib().cox_grid_broadcast(op, dt, d_in, d_out, n, d_ws, ws_bytes, stream)


def cox_grid_broadcast_workspace(n) -> int:
    return lib().cox_grid_broadcast_workspace(n)


def cox_coalesced(fn, dt, block_dim, d_in, d_active, d_out, n, param, stream) -> int:
    return lib().cox_coalesced(fn, dt, block_dim, d_in, d_active, d_out, n, param, stream)


def cox_filter_aggregated(dt, d_keys, n, threshold, d_out, d_count, stream) -> int:
    return lib().cox_filter_aggregated(dt, d_keys, n, threshold, d_out, d_count, stream)


def cox_vote_stats(dt, width, d_pred, n, seg_len, d_stats, stream) -> int:
    return lib().cox_vote_stats(dt, width, d_pred, n, seg_len, d_stats, stream)


def cox_integral_image(in_dt, batch, height, width, d_in, d_out, d_ws, ws_bytes, stream) -> int:
    return lib().cox_integral_image(in_dt, batch, height, width, d_in, d_out, d_ws, ws_bytes, stream)


def cox_integral_image_workspace(batch, height, width) -> int:
    return lib().cox_integral_image_workspace(batch, height, width)


def cox_ballot_compact(dt, width, block_dim, d_keys, n, threshold, d_out, d_count, d_ws, ws_bytes, flags,
                       stream) -> int:
    return lib().cox_ballot_compact(dt, width, block_dim, d_keys, n, threshold, d_out, d_count, d_ws, ws_bytes,
                                    flags, stream)


def cox_ballot_compact_workspace(n, block_dim) -> int:
    return lib().cox_ballot_compact_workspace(n, block_dim)


def cox_ballot_compact_static(dt, width, block_dim, d_keys, n, threshold, d_out, d_count, stream) -> int:
    return lib().cox_ballot_compact_static(dt, width, block_dim, d_keys, n, threshold, d_out, d_count, stream)


COX_COMPACT_STATIC_SCRATCH_BYTES = 1 << 20


def cox_match_histogram(dt, width, block_dim, d_keys, n, bins, d_hist, d_ignored, flags, stream) -> int:
    return lib().cox_match_histogram(dt, width, block_dim, d_keys, n, bins, d_hist, d_ignored, flags, stream)


class cox_batch_tune(ctypes.Structure):
    """Launch shape of the batched kernel (mirrors the C struct; ept defaults to 8)."""
    _fields_ = [("block_dim", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("width", ctypes.c_int),
                ("fp64_segments", ctypes.c_int), ("native_match", ctypes.c_int), ("ept", ctypes.c_int)]

    def __init__(self, block_dim=0, ctas_per_sm=0, width=0, fp64_segments=0, native_match=0, ept=8):
        super().__init__(block_dim, ctas_per_sm, width, fp64_segments, native_match, ept)

    def astuple(self):
        return (self.block_dim, self.ctas_per_sm, self.width, self.fp64_segments, self.native_match, self.ept)


def cox_batch_workspace(num_arrays) -> int:
    return lib().cox_batch_workspace(num_arrays)


def cox_batch_prepare(num_arrays, h_lens, d_ws, ws_bytes, stream) -> int:
    return lib().cox_batch_prepare(num_arrays, h_lens, d_ws, ws_bytes, stream)


def cox_batch_sum_hist(num_arrays, d_vals, d_keys, tune, d_ws, ws_bytes, d_sums, d_sums64, d_hists, stream) -> int:
    return lib().cox_batch_sum_hist(num_arrays, d_vals, d_keys, tune, d_ws, ws_bytes, d_sums, d_sums64, d_hists,
                                    stream)


def cox_batch_percall_scratch(max_len) -> int:
    return lib().cox_batch_percall_scratch(max_len)


def cox_batch_percall(num_arrays, h_vals, h_keys, h_lens, d_sums, d_hists, d_scratch, scratch_bytes, events,
                      stream) -> int:
    return lib().cox_batch_percall(num_arrays, h_vals, h_keys, h_lens, d_sums, d_hists, d_scratch, scratch_bytes,
                                   events, stream)


def cox_batch_graph_create(num_arrays, d_vals, d_keys, tune, d_ws, ws_bytes, d_sums, d_sums64, d_hists, out) -> int:
    return lib().cox_batch_graph_create(num_arrays, d_vals, d_keys, tune, d_ws, ws_bytes, d_sums, d_sums64, d_hists,
                                        out)


def cox_graph_launch(g, stream) -> int:
    return lib().cox_graph_launch(g, stream)


def cox_graph_destroy(g) -> None:
    lib().cox_graph_destroy(g)


def cox_batch_autotune(num_arrays, d_vals, d_keys, d_ws, ws_bytes, d_sums, d_hists, reps, cache_path, best, best_ms,
                       stream) -> int:
    return lib().cox_batch_autotune(num_arrays, d_vals, d_keys, d_ws, ws_bytes, d_sums, d_hists, reps, cache_path,
                                    best, best_ms, stream)


def cox_batch_tune_lookup(cache_path, num_arrays, total_elems, tune) -> int:
    return lib().cox_batch_tune_lookup(cache_path, num_arrays, total_elems, tune)


def cox_device_status(stream) -> int:
    return lib().cox_device_status(stream)


def cox_set_spin_limit(polls: int) -> None:
    lib().cox_set_spin_limit(polls)


# ------------------------------------------------------------ tensor helpers
def _torch():
    import torch
    return torch


def _check(status: int, what: str):
    if status != COX_OK:
        raise CoxError(status, what)


def _stream(dev):
    return _torch().cuda.current_stream(dev).cuda_stream


def _dtype_code(x, unsigned: bool = False) -> int:
    t = _torch()
    if x.dtype == t.float32:
        return COX_F32
    if x.dtype == t.int32:
        return COX_U32 if unsigned else COX_I32
    if hasattr(t, "uint32") and x.dtype == t.uint32:
        return COX_U32
    raise TypeError(f"32-bit int or float tensor required, got {x.dtype}")


def _dev_tensor(x):
    if not x.is_cuda:
        raise ValueError("CUDA tensor required")
    if not x.is_contiguous():
        raise ValueError("contiguous tensor required")
    return x


def shfl(fn: int, x, width: int = 32, block_dim: int = 256, param: int = 0, unsigned: bool = False, out=None):
    """One warp function per lane (cox_shfl).  Masks come back as int32 bit patterns."""
    t = _torch()
    x = _dev_tensor(x)
    dt = _dtype_code(x, unsigned)
    if out is None:
        out = t.empty_like(x) if fn <= COX_SHFL_XOR else t.empty(x.shape, dtype=t.int32, device=x.device)
    _check(cox_shfl(fn, dt, width, block_dim, x.data_ptr(), out.data_ptr(), x.numel(), param, FULL_MASK,
                    _stream(x.device)), "cox_shfl")
    return out


def reduce_out_len(scope: int, n: int, width: int, block_dim: int) -> int:
    if scope == COX_SCOPE_TILE:
        return -(-n // width)
    if scope == COX_SCOPE_BLOCK:
        return -(-n // block_dim)
    return 1


def tile_reduce(x, op: int = COX_SUM, width: int = 32, block_dim: int = 256, scope: int = COX_SCOPE_BLOCK,
                compensated: bool = False, fp64_combine: bool = False, unsigned: bool = False, with_lo: bool = False,
                workspace=None, out=None):
    """Tile/block/grid reduction (cox_tile_reduce).  Returns out, or (out, lo) with with_lo."""
    t = _torch()
    x = _dev_tensor(x)
    n = x.numel()
    m = reduce_out_len(scope, n, width, block_dim)
    if out is None:
        out = t.empty(m, dtype=x.dtype, device=x.device)
    lo = t.zeros(m, dtype=t.float32, device=x.device) if with_lo else None
    flags = (COX_F_COMPENSATED if compensated else 0) | (COX_F_FP64_COMBINE if fp64_combine else 0)
    ws_bytes = cox_tile_reduce_workspace(scope, n, block_dim)
    if ws_bytes and workspace is None:
        workspace = t.empty(ws_bytes, dtype=t.uint8, device=x.device)
    _check(cox_tile_reduce(op, _dtype_code(x, unsigned), width, block_dim, scope, x.data_ptr(), out.data_ptr(), n,
                           flags, lo.data_ptr() if lo is not None else None,
                           workspace.data_ptr() if workspace is not None else None, ws_bytes,
                           _stream(x.device)), "cox_tile_reduce")
    return (out, lo) if with_lo else out


def tile_scan(x, op: int = COX_SUM, width: int = 32, block_dim: int = 256, compensated: bool = False,
              unsigned: bool = False, out=None):
    """Tile inclusive scan (cox_tile_scan)."""
    t = _torch()
    x = _dev_tensor(x)
    if out is None:
        out = t.empty_like(x)
    _check(cox_tile_scan(op, _dtype_code(x, unsigned), width, block_dim, x.data_ptr(), out.data_ptr(), x.numel(),
                         COX_F_COMPENSATED if compensated else 0, _stream(x.device)), "cox_tile_scan")
    return out


def scan(x, op: int = COX_SUM, scope: int = COX_SCOPE_GRID, block_dim: int = 256, compensated: bool = False,
         exclusive: bool = False, unsigned: bool = False, out=None, workspace=None):
    """Block- or grid-scope inclusive/exclusive scan (cox_scan)."""
    t = _torch()
    x = _dev_tensor(x)
    if out is None:
        out = t.empty_like(x)
    ws_bytes = cox_scan_workspace(scope, x.numel())
    if ws_bytes and workspace is None:
        workspace = t.empty(ws_bytes, dtype=t.uint8, device=x.device)
    _check(cox_scan(op, _dtype_code(x, unsigned), scope, block_dim, x.data_ptr(), out.data_ptr(), x.numel(),
                    COX_F_COMPENSATED if compensated else 0, 1 if exclusive else 0,
                    workspace.data_ptr() if workspace is not None else None, ws_bytes, _stream(x.device)),
           "cox_scan")
    return out


def grid_broadcast(x, op: int = COX_GRID_SUB_MIN, unsigned: bool = False, out=None, workspace=None):
    """Reduce-then-broadcast in one cooperative kernel (cox_grid_broadcast)."""
    t = _torch()
    x = _dev_tensor(x)
    if out is None:
        out = t.empty_like(x)
    ws_bytes = cox_grid_broadcast_workspace(x.numel())
    if workspace is None:
        workspace = t.empty(ws_bytes, dtype=t.uint8, device=x.device)
    _check(cox_grid_broadcast(op, _dtype_code(x, unsigned), x.data_ptr(), out.data_ptr(), x.numel(),
                              workspace.data_ptr(), ws_bytes, _stream(x.device)), "cox_grid_broadcast")
    return out


def ballot_compact(keys, threshold: int, width: int = 32, block_dim: int = 256, unsigned: bool = False,
                   workspace=None, out=None, count=None):
    """Stable compaction of keys < threshold (cox_ballot_compact).  Returns (out, count) device tensors."""
    t = _torch()
    keys = _dev_tensor(keys)
    n = keys.numel()
    if out is None:
        out = t.empty(max(n, 1), dtype=keys.dtype, device=keys.device)
    if count is None:
        count = t.empty(1, dtype=t.int64, device=keys.device)
    ws_bytes = cox_ballot_compact_workspace(n, block_dim)
    if workspace is None:
        workspace = t.empty(max(ws_bytes, 16), dtype=t.uint8, device=keys.device)
    _check(cox_ballot_compact(COX_U32 if unsigned else COX_I32, width, block_dim, keys.data_ptr(), n, int(threshold),
                              out.data_ptr(), count.data_ptr(), workspace.data_ptr(), workspace.numel(), 0,
                              _stream(keys.device)), "cox_ballot_compact")
    return out, count


def match_histogram(keys, bins: int = 256, width: int = 32, block_dim: int = 256, unsigned: bool = False,
                    native_match: bool = False, direct: bool = False, ballot_match: bool = False):
    """Match-any histogram (cox_match_histogram).  Returns (hist int32[bins], ignored int64[1])."""
    t = _torch()
    keys = _dev_tensor(keys)
    hist = t.empty(bins, dtype=t.int32, device=keys.device)
    ign = t.empty(1, dtype=t.int64, device=keys.device)
    _check(cox_match_histogram(COX_U32 if unsigned else COX_I32, width, block_dim, keys.data_ptr(), keys.numel(),
                               bins, hist.data_ptr(), ign.data_ptr(),
                               (COX_F_NATIVE_MATCH if native_match else 0) | (COX_F_DIRECT_ATOMICS if direct else 0)
                               | (COX_F_BALLOT_MATCH if ballot_match else 0), _stream(keys.device)),
           "cox_match_histogram")
    return hist, ign


def device_status(stream=None) -> int:
    """Synchronise and read/clear the device status word (cox_device_status)."""
    return cox_device_status(stream if stream is not None else _stream(None))


class Batch:
    """A prepared batch of uneven arrays for cox_batch_sum_hist.

    `vals` / `keys`: lists of 1-D CUDA tensors (float32 values, int32 keys),
    array a being vals[a] with keys[a] of the same length.  Holds the device
    pointer tables, the workspace and the outputs (sums fp32, sums64 fp64,
    hists int32 [A, 256]); run() enqueues one batched call, graph() captures
    one into a CUDA graph for replay.
    """

    def __init__(self, vals, keys, tune=None):
        t = _torch()
        if len(vals) != len(keys) or not vals:
            raise ValueError("vals and keys must be non-empty lists of the same length")
        dev = vals[0].device
        self.A = len(vals)
        self.vals, self.keys = vals, keys  # keep the tensors alive
        lens = [int(v.numel()) for v in vals]
        for v, k in zip(vals, keys):
            if v.numel() != k.numel() or v.dtype != t.float32 or k.dtype != t.int32:
                raise ValueError("each array needs float32 values and int32 keys of equal length")
        self.lens = t.tensor(lens, dtype=t.int64)
        self.total = sum(lens)
        self.pv = t.tensor([v.data_ptr() for v in vals], dtype=t.int64, device=dev)
        self.pk = t.tensor([k.data_ptr() for k in keys], dtype=t.int64, device=dev)
        self.ws_bytes = cox_batch_workspace(self.A)
        self.ws = t.empty(self.ws_bytes, dtype=t.uint8, device=dev)
        self.sums = t.empty(self.A, dtype=t.float32, device=dev)
        self.sums64 = t.empty(self.A, dtype=t.float64, device=dev)
        self.hists = t.empty((self.A, 256), dtype=t.int32, device=dev)
        self.tune = None
        if tune is not None:
            self.tune = cox_batch_tune(*tune) if not isinstance(tune, cox_batch_tune) else tune
        self.stream = _stream(dev)
        _check(cox_batch_prepare(self.A, self.lens.data_ptr(), self.ws.data_ptr(), self.ws_bytes, self.stream),
               "cox_batch_prepare")

    def _tune_ptr(self):
        return ctypes.addressof(self.tune) if self.tune is not None else None

    def run(self, stream=None):
        _check(cox_batch_sum_hist(self.A, self.pv.data_ptr(), self.pk.data_ptr(), self._tune_ptr(),
                                  self.ws.data_ptr(), self.ws_bytes, self.sums.data_ptr(), self.sums64.data_ptr(),
                                  self.hists.data_ptr(), stream if stream is not None else self.stream),
               "cox_batch_sum_hist")
        return self.sums, self.sums64, self.hists

    def graph(self):
        g = ctypes.c_void_p()
        _check(cox_batch_graph_create(self.A, self.pv.data_ptr(), self.pk.data_ptr(), self._tune_ptr(),
                                      self.ws.data_ptr(), self.ws_bytes, self.sums.data_ptr(), self.sums64.data_ptr(),
                                      self.hists.data_ptr(), ctypes.byref(g)), "cox_batch_graph_create")
        return Graph(g)

    def autotune(self, reps: int = 3, cache_path=None):
        best = cox_batch_tune()
        ms = ctypes.c_float()
        _check(cox_batch_autotune(self.A, self.pv.data_ptr(), self.pk.data_ptr(), self.ws.data_ptr(), self.ws_bytes,
                                  self.sums.data_ptr(), self.hists.data_ptr(), reps,
                                  cache_path.encode() if cache_path else None, ctypes.byref(best), ctypes.byref(ms),
                                  self.stream), "cox_batch_autotune")
        self.tune = best
        return best, ms.value


class Graph:
    """An instantiated CUDA graph from the library (cox_graph)."""

    def __init__(self, handle):
        self.handle = handle

    def launch(self, stream=None):
        _check(cox_graph_launch(self.handle, stream if stream is not None else _stream(None)), "cox_graph_launch")

    def __del__(self):
        try:
            if self.handle:
                cox_graph_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


# ------------------------------------------------------------------ server
COX_REQ_REDUCE, COX_REQ_SCAN, COX_REQ_COMPACT = 0, 1, 2


class cox_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("dt", ctypes.c_int), ("width", ctypes.c_int), ("flags", ctypes.c_uint),
                ("n", ctypes.c_int64), ("threshold", ctypes.c_int64), ("d_in", ctypes.c_void_p)]


class cox_trace_item(ctypes.Structure):
    _fields_ = [("arrival_s", ctypes.c_double), ("req", cox_request)]


class cox_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("max_batch", ctypes.c_int64), ("budget_bytes", ctypes.c_size_t),
                ("used_bytes", ctypes.c_size_t), ("peak_bytes", ctypes.c_size_t), ("queued", ctypes.c_int64),
                ("wait_s", ctypes.c_double), ("run_s", ctypes.c_double)]

    def asdict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def make_request(kind: int, x, width: int = 32, compensated: bool = False, threshold: int = 0,
                 unsigned: bool = False, n: int | None = None) -> cox_request:
    """A cox_request over the CUDA tensor x (its first n elements)."""
    t = _torch()
    x = _dev_tensor(x)
    if kind == COX_REQ_COMPACT:
        dt = COX_U32 if unsigned else COX_I32
    else:
        dt = COX_F32 if x.dtype == t.float32 else COX_I32
    return cox_request(kind, dt, width, COX_F_COMPENSATED if compensated else 0,
                       x.numel() if n is None else int(n), int(threshold), x.data_ptr())


class _DevView:
    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 2}


class Server:
    """Continuous-batching request server (cox_server_*) over a device arena."""

    def __init__(self, budget_bytes: int, max_requests: int = 1024):
        self.handle = ctypes.c_void_p()
        _check(lib().cox_server_create(int(budget_bytes), int(max_requests), ctypes.byref(self.handle)),
               "cox_server_create")
        self._keep = {}

    def submit(self, req: cox_request, keep=None) -> int:
        t = ctypes.c_uint64()
        _check(lib().cox_server_submit(self.handle, ctypes.byref(req), ctypes.byref(t)), "cox_server_submit")
        if keep is not None:
            self._keep[t.value] = keep
        return t.value

    def submit_many(self, reqs, keep=None) -> list:
        """Queues the requests together (cox_server_submit_many); keep[i] is
        held for reqs[i] until it is released."""
        arr = (cox_request * len(reqs))(*reqs)
        ts = (ctypes.c_uint64 * len(reqs))()
        _check(lib().cox_server_submit_many(self.handle, arr, len(reqs), ts), "cox_server_submit_many")
        if keep is not None:
            for t, k in zip(ts, keep):
                self._keep[t] = k
        return list(ts)

    def poll(self, ticket: int) -> bool:
        d = ctypes.c_int()
        _check(lib().cox_server_poll(self.handle, ticket, ctypes.byref(d)), "cox_server_poll")
        return bool(d.value)

    def wait(self, ticket: int, timeout_s: float = 30.0) -> None:
        _check(lib().cox_server_wait(self.handle, ticket, float(timeout_s)), "cox_server_wait")

    def result(self, ticket: int, req: cox_request):
        """A copy (torch CUDA tensor) of a done request's output."""
        t = _torch()
        p = ctypes.c_void_p()
        c = ctypes.c_int64()
        _check(lib().cox_server_result(self.handle, ticket, ctypes.byref(p), ctypes.byref(c)), "cox_server_result")
        if req.kind == COX_REQ_REDUCE:
            n, typ = 2, ("<f4" if req.dt == COX_F32 else "<i4")
        else:
            n, typ = c.value, ("<f4" if req.dt == COX_F32 else "<i4")
        if n == 0:
            return t.empty(0, dtype=t.float32 if typ == "<f4" else t.int32, device="cuda")
        return t.as_tensor(_DevView(p.value, n, typ), device="cuda").clone()

    def release(self, ticket: int) -> None:
        _check(lib().cox_server_release(self.handle, ticket), "cox_server_release")
        self._keep.pop(ticket, None)

    def stats(self) -> dict:
        st = cox_server_stats()
        _check(lib().cox_server_get_stats(self.handle, ctypes.byref(st)), "cox_server_get_stats")
        return st.asdict()

    def run_trace(self, items):
        """Replays (arrival_s, cox_request) pairs; returns (latencies list, wall seconds)."""
        arr = (cox_trace_item * len(items))(*[cox_trace_item(a, r) for a, r in items])
        lat = (ctypes.c_double * len(items))()
        wall = ctypes.c_double()
        _check(lib().cox_server_run_trace(self.handle, arr, len(items), lat, ctypes.byref(wall)),
               "cox_server_run_trace")
        return list(lat), wall.value

    def close(self):
        if self.handle:
            lib().cox_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def percall_run_trace(items, scratch=None):
    """The same trace with one launch per request (cox_percall_run_trace)."""
    t = _torch()
    max_n = max(r.n for _, r in items)
    need = lib().cox_percall_scratch(max_n)
    if scratch is None:
        scratch = t.empty(need, dtype=t.uint8, device="cuda")
    arr = (cox_trace_item * len(items))(*[cox_trace_item(a, r) for a, r in items])
    lat = (ctypes.c_double * len(items))()
    wall = ctypes.c_double()
    _check(lib().cox_percall_run_trace(arr, len(items), scratch.data_ptr(), scratch.numel(), lat,
                                       ctypes.byref(wall)), "cox_percall_run_trace")
    return list(lat), wall.value
