"""CPU oracle of the warp-collective library -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never does, and this
package imports nothing from it: the two share only the seeded input
generators.

Thin numpy wrapper over ``liboracle.so`` (built from ``cox_oracle.cpp`` by
``oracle/build.py``), a collapsed-loop executor of CUDA warp-function
semantics: inter-warp loops around intra-warp loops over per-lane register
arrays, each warp function a write phase and a read phase on an exchange array
(Sections 2.3, 3.2 and 3.6 of the paper), one CUDA block per task on a CPU
thread pool (Section 4).  Each function's docstring names the passage it
follows; the C source carries the details.

Codes (this package's own numbering, equal by value to the library's ABI):
dtype I32=0 U32=1 F32=2; op SUM=0 MIN=1 MAX=2 AND=3 OR=4 XOR=5;
warp function SHFL_IDX=0 SHFL_UP=1 SHFL_DOWN=2 SHFL_XOR=3 BALLOT=4 ANY=5 ALL=6
MATCH_ANY=7; scope TILE=0 BLOCK=1 GRID=2.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import build as _build, lib_path

I32, U32, F32 = 0, 1, 2
SUM, MIN, MAX, AND, OR, XOR = 0, 1, 2, 3, 4, 5
SHFL_IDX, SHFL_UP, SHFL_DOWN, SHFL_XOR, BALLOT, ANY, ALL, MATCH_ANY = range(8)
TILE, BLOCK, GRID = 0, 1, 2

_lib = None
_P = ctypes.c_void_p
_I64 = ctypes.c_int64


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        _build()
    lib = ctypes.CDLL(path)
    sig = {
        "oracle_set_threads": (None, [ctypes.c_int]),
        "oracle_threads": (ctypes.c_int, []),
        "oracle_debug_fuse_phases": (None, [ctypes.c_int]),
        "oracle_shfl": (ctypes.c_int, [ctypes.c_int] * 4 + [_P, _P, _I64, ctypes.c_int]),
        "oracle_code1": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P]),
        "oracle_code4": (ctypes.c_int, [ctypes.c_int, _P]),
        "oracle_vote_pair": (ctypes.c_int, [ctypes.c_int, _P]),
        "oracle_reduce_emulate": (ctypes.c_int, [ctypes.c_int] * 6 + [_P, _P, _P, _I64]),
        "oracle_reduce_counts": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _I64, _P]),
        "oracle_reduce_ref": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _I64, _P, _I64, _P, _P, _P]),
        "oracle_scan_emulate": (ctypes.c_int, [ctypes.c_int] * 5 + [_P, _P, _I64]),
        "oracle_coalesced": (ctypes.c_int, [ctypes.c_int] * 3 + [_P, _P, _P, _I64, ctypes.c_int]),
        "oracle_scan_ref": (ctypes.c_int, [ctypes.c_int] * 3 + [_P, _I64, _P, _P, _P]),
        "oracle_ballot_compact": (ctypes.c_int, [ctypes.c_int] * 3 + [_P, _I64, _I64, _P, _P]),
        "oracle_match_histogram": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, _I64, ctypes.c_int, _P, _P]),
        "oracle_batch_ref": (ctypes.c_int, [_I64, _P, _P, _P, ctypes.c_int, _P, _P, _P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _bits(x: np.ndarray) -> np.ndarray:
    """View a 32-bit array as uint32 bit patterns (contiguous)."""
    x = np.ascontiguousarray(x)
    if x.dtype.itemsize != 4:
        raise TypeError(f"32-bit elements required, got {x.dtype}")
    return x.view(np.uint32)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"{what}: oracle status {rc}")


_NP = {I32: np.int32, U32: np.uint32, F32: np.float32}


def set_threads(k: int) -> None:
    """Size of the CPU thread pool that runs blocks (0 = one per hardware thread)."""
    _load().oracle_set_threads(int(k))


def threads() -> int:
    return int(_load().oracle_threads())


def debug_fuse_phases(on: bool) -> None:
    """Planted-mistake switch: drop the RAW/WAR warp barriers of Section 3.2."""
    _load().oracle_debug_fuse_phases(1 if on else 0)


def shfl(fn: int, dt: int, width: int, block_dim: int, x: np.ndarray, param: int = 0) -> np.ndarray:
    """Warp functions of Section 2.2.1 (Code 1: shfl_down; Code 4: all) on every lane.

    Shuffles return the source lane's value (0 if that lane is padding);
    BALLOT/MATCH_ANY give tile-local uint32 masks; ANY/ALL give int32 0/1.
    """
    xb = _bits(x)
    out = np.zeros(xb.size, np.uint32)
    _check(_load().oracle_shfl(fn, dt, width, block_dim, _ptr(xb), _ptr(out), xb.size, int(param)), "shfl")
    if fn <= SHFL_XOR:
        return out.view(_NP[dt])
    if fn in (BALLOT, MATCH_ANY):
        return out
    return out.view(np.int32)


def code1(block_dim: int, mode: int = 0) -> np.ndarray:
    """Code 1 (Section 2.3) on one block with all-ones input; mode 1 = Code 3's CPU rule."""
    out = np.zeros(block_dim, np.int32)
    _check(_load().oracle_code1(block_dim, mode, _ptr(out)), "code1")
    return out


def code4(block_dim: int) -> np.ndarray:
    """Code 4 (Section 3.1): result[tx] = __all_sync(-1, tx % 2)."""
    out = np.zeros(block_dim, np.int32)
    _check(_load().oracle_code4(block_dim, _ptr(out)), "code4")
    return out


def vote_pair(block_dim: int) -> np.ndarray:
    """Two consecutive votes (all(tx%2), then all(1)) through one exchange array (Code 5)."""
    out = np.zeros(2 * block_dim, np.int32)
    _check(_load().oracle_vote_pair(block_dim, _ptr(out)), "vote_pair")
    return out.reshape(block_dim, 2)


def n_out(scope: int, n: int, width: int, block_dim: int) -> int:
    if scope == TILE:
        return -(-n // width)
    if scope == BLOCK:
        return -(-n // block_dim)
    return 1 if n > 0 else 0


def reduce_emulate(op: int, dt: int, width: int, block_dim: int, scope: int, x: np.ndarray,
                   compensated: bool = False):
    """Tile/block reduction in the kernels' association order (Code 1 tree + block combine).

    Returns (out, lo); lo is the compensated result's low word (zeros otherwise).
    """
    xb = _bits(x)
    m = n_out(scope, xb.size, width, block_dim)
    out = np.zeros(m, np.uint32)
    lo = np.zeros(m, np.float32)
    _check(_load().oracle_reduce_emulate(op, dt, width, block_dim, scope, int(compensated),
                                         _ptr(xb), _ptr(out), _ptr(lo), xb.size), "reduce_emulate")
    return out.view(_NP[dt]), lo


def reduce_counts(width: int, block_dim: int, n: int) -> np.ndarray:
    """Appendix A instrumentation: [3, grid*block] statement counts per thread."""
    grid = -(-n // block_dim)
    out = np.zeros(3 * grid * block_dim, np.int32)
    _check(_load().oracle_reduce_counts(width, block_dim, n, _ptr(out)), "reduce_counts")
    return out.reshape(3, grid * block_dim)


def reduce_ref(op: int, dt: int, seg_len: int, x: np.ndarray):
    """Plain definition of the reduction over segments of seg_len elements.

    Returns (bits, ref64, abs64): exact bits for integer ops and fp32 min/max,
    FP64 Neumaier value and sum |x| for fp32 sums.
    """
    xb = _bits(x)
    m = -(-xb.size // seg_len) if xb.size else 0
    bits = np.zeros(m, np.uint32)
    ref = np.zeros(m, np.float64)
    ab = np.zeros(m, np.float64)
    _check(_load().oracle_reduce_ref(op, dt, seg_len, _ptr(xb), xb.size, _ptr(bits), _ptr(ref), _ptr(ab)),
           "reduce_ref")
    return bits.view(_NP[dt]), ref, ab


def scan_emulate(op: int, dt: int, width: int, block_dim: int, x: np.ndarray,
                 compensated: bool = False) -> np.ndarray:
    """Tile inclusive scan by Hillis-Steele on shfl_up (SDK shfl_scan_test, Table 1)."""
    xb = _bits(x)
    out = np.zeros(xb.size, np.uint32)
    _check(_load().oracle_scan_emulate(op, dt, width, block_dim, int(compensated), _ptr(xb), _ptr(out),
                                       xb.size), "scan_emulate")
    return out.view(_NP[dt])


def scan_ref(op: int, dt: int, width: int, x: np.ndarray):
    """Plain definition of the tile inclusive scan (segments of `width` elements)."""
    xb = _bits(x)
    bits = np.zeros(xb.size, np.uint32)
    ref = np.zeros(xb.size, np.float64)
    ab = np.zeros(xb.size, np.float64)
    _check(_load().oracle_scan_ref(op, dt, width, _ptr(xb), xb.size, _ptr(bits), _ptr(ref), _ptr(ab)),
           "scan_ref")
    return bits.view(_NP[dt]), ref, ab


def ballot_compact(dt: int, width: int, block_dim: int, keys: np.ndarray, threshold: int):
    """Ballot-driven stable compaction (filter_arr, Table 1): keys with key < threshold."""
    kb = _bits(keys)
    out = np.zeros(kb.size, np.uint32)
    cnt = np.zeros(1, np.int64)
    _check(_load().oracle_ballot_compact(dt, width, block_dim, _ptr(kb), kb.size, int(threshold), _ptr(out),
                                         _ptr(cnt)), "ballot_compact")
    c = int(cnt[0])
    return out[:c].view(_NP[dt]).copy(), c


def match_histogram(width: int, block_dim: int, keys: np.ndarray, bins: int = 256):
    """Match-any histogram: leader of each peer group adds the group size."""
    kb = np.ascontiguousarray(keys, dtype=np.int32)
    hist = np.zeros(bins, np.int32)
    ign = np.zeros(1, np.int64)
    _check(_load().oracle_match_histogram(width, block_dim, _ptr(kb), kb.size, bins, _ptr(hist), _ptr(ign)),
           "match_histogram")
    return hist, int(ign[0])


def batch_ref(offsets: np.ndarray, vals: np.ndarray, keys: np.ndarray, bins: int = 256):
    """Per array: FP64 Neumaier sum, sum |x|, and the bins-bin key histogram."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    vals = np.ascontiguousarray(vals, dtype=np.float32)
    keys = np.ascontiguousarray(keys, dtype=np.int32)
    a = offsets.size - 1
    sums = np.zeros(a, np.float64)
    ab = np.zeros(a, np.float64)
    hists = np.zeros((a, bins), np.int32)
    _check(_load().oracle_batch_ref(a, _ptr(offsets), _ptr(vals), _ptr(keys), bins, _ptr(sums), _ptr(ab),
                                    _ptr(hists)), "batch_ref")
    return sums, ab, hists


def rel_err(y: np.ndarray, ref64: np.ndarray, abs64: np.ndarray) -> np.ndarray:
    """Error metric for fp32 sums: |y - r| / max(|r|, u * sum|x|), u = 2^-24.

    The plain relative error |y - r| / |r| is undefined where the reference
    sum cancels to (near) zero; the floor u * sum|x| is the size of one fp32
    rounding of the inputs that feed the result.
    """
    y = np.asarray(y, dtype=np.float64)
    den = np.maximum(np.abs(ref64), 2.0 ** -24 * abs64)
    den = np.where(den == 0, 1.0, den)
    return np.abs(y - ref64) / den


# ------------------------------------------- grid-wide reduce-then-broadcast
# The cooperative-groups grid sync that gpuConjugateGradient needs and COX
# cannot provide (Table 1; Section 5.1): a reduction over the whole grid,
# a grid-wide barrier, then every thread uses the result.  The oracle is the
# plain definition of the two steps, with no barrier to model.
GRID_SUB_MIN, GRID_NORMALIZE = 0, 1


def fp32_min_total_order(x: np.ndarray) -> np.float32:
    """The minimum of fp32 values under IEEE totalOrder restricted to numbers
    (-0 < +0), NaNs ignored; NaN if every value is NaN."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    key = np.where(u & 0x80000000, ~u, u | 0x80000000).astype(np.uint32)
    key = np.where(np.isnan(x), np.uint32(0xFFFFFFFF), key)
    k = key.min()
    bits = np.uint32(~k) if not (k & 0x80000000) else np.uint32(k & 0x7FFFFFFF)
    if k == 0xFFFFFFFF:
        bits = np.uint32(0x7FFFFFFF)
    return np.array([bits], np.uint32).view(np.float32)[0]


def grid_sub_min(dt: int, x: np.ndarray) -> np.ndarray:
    """y_i = x_i - min_j x_j: integers wrap mod 2^32 (reading R6); fp32 is one
    IEEE round-to-nearest subtraction of the minimum taken in totalOrder
    (-0 below +0, NaNs ignored; reading R18)."""
    if dt == F32:
        x = np.ascontiguousarray(x, dtype=np.float32)
        with np.errstate(invalid="ignore"):
            return (x - fp32_min_total_order(x)).astype(np.float32)
    t = np.int32 if dt == I32 else np.uint32
    x = np.ascontiguousarray(x).view(t)
    m = np.array([x.min()], dtype=t).view(np.uint32)
    return (x.view(np.uint32) - m).view(t)


def grid_normalize_ref(x: np.ndarray):
    """y_i = x_i / sqrt(sum_j x_j^2) in FP64 for fp32 x.  Squares of fp32
    values are exact in FP64 and math.fsum rounds their sum once, so the
    norm is the correctly rounded FP64 value.  Returns (ref64, norm64)."""
    import math
    x64 = np.ascontiguousarray(x, dtype=np.float32).astype(np.float64)
    norm = math.sqrt(math.fsum((x64 * x64).tolist()))
    return x64 / norm, norm


# ------------------------------------------------ coalesced groups (dynamic)
CG_SIZE, CG_RANK, CG_SHFL, CG_SHFL_UP, CG_SHFL_DOWN, CG_BALLOT, CG_ANY, CG_ALL, CG_REDUCE_SUM, CG_SCAN_SUM = range(10)


def coalesced(fn: int, dt: int, block_dim: int, x: np.ndarray, active: np.ndarray, param: int = 0) -> np.ndarray:
    """Warp functions over coalesced_threads() groups (Section 2.2.2's dynamic
    groups; Section 2.2.3's runtime masks): the group of a warp is its lanes
    with active != 0, in lane order.  Returns (out, written): out[i] for the
    active lanes; written marks them (inactive lanes get no result)."""
    xb = _bits(x)
    act = np.ascontiguousarray(active, dtype=np.int32)
    out = np.zeros(xb.size, np.uint32)
    _check(_load().oracle_coalesced(fn, dt, block_dim, _ptr(xb), _ptr(act), _ptr(out), xb.size, param),
           "coalesced")
    return out, act != 0


def filter_multiset(dt: int, keys: np.ndarray, threshold: int):
    """The keys an unordered filter keeps (key < threshold in the keys' own
    signedness; threshold clamped to the key range, reading R11), sorted, and
    their count: what filter_arr's aggregated-atomic output holds in some order."""
    k = np.ascontiguousarray(keys).view(np.int32 if dt == I32 else np.uint32).astype(np.int64)
    kept = np.sort(k[k < threshold])
    return kept, int(kept.size)


# ------------------------------------- vote statistics and integral images
def vote_stats(width: int, pred: np.ndarray, seg_len: int) -> np.ndarray:
    """Batched statistics of the vote kernels (VoteAny/VoteAll, Table 1): the
    array is cut into segments of seg_len elements (a multiple of width; the
    last may be shorter), each segment into tiles of `width` lanes; per
    segment: [tiles whose any() is true, tiles whose all() is true, true
    predicates].  A ragged last tile's missing lanes are padding with a false
    predicate (reading R5), so its all() is false.  Predicate: value != 0."""
    p = np.ascontiguousarray(pred).view(np.int32) != 0
    n = p.size
    nseg = (n + seg_len - 1) // seg_len
    out = np.zeros((nseg, 3), np.int64)
    for s in range(nseg):
        seg = p[s * seg_len:min(n, (s + 1) * seg_len)]
        t = (seg.size + width - 1) // width
        padded = np.zeros(t * width, bool)
        padded[:seg.size] = seg
        tiles = padded.reshape(t, width)
        out[s] = [tiles.any(axis=1).sum(), tiles.all(axis=1).sum(), seg.sum()]
    return out


def integral_image(img: np.ndarray) -> np.ndarray:
    """Integral images of a batch (B, H, W) of uint8 or 32-bit images:
    I[b, y, x] = sum over y' <= y, x' <= x of img[b, y', x'], mod 2^32 (the
    SDK's shfl_intimage_rows / shfl_vertical_shfl pair, Table 1, reading R6)."""
    a = np.asarray(img)
    a = a.astype(np.uint64) if a.dtype == np.uint8 else a.view(np.uint32).astype(np.uint64)
    return (np.cumsum(np.cumsum(a, axis=2), axis=1) % (1 << 32)).astype(np.uint32)
