"""Pins of the CPU oracle against things other than itself.

Each test fixes one oracle function by the paper's printed values (Code 1,
Code 4 of the paper, in tests/golden), by brute-force lane enumeration
(tests/lanes.py), by numpy/math library routines that compute the plain
definition (np.add.reduceat, np.cumsum, boolean masks, np.bincount,
math.fsum), by closed forms, or by the invariants of each op.  A planted
mistake (the oracle's debug switch that drops the warp barriers of
Section 3.2) must fail the paper pins.
"""
import math
import os

import numpy as np
import pytest

import oracle as o
from paper_2112_10034_gb300 import inputs
from tests import lanes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
WIDTHS = [2, 4, 8, 16, 32]


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([int(t) for t in line.split()])
    return rows


# ------------------------------------------------------------ paper pins
def test_code1_golden_lane0_is_32():
    for block, lane, value in _golden("code1_shfl_down.txt"):
        for mode in (0, 1):
            assert o.code1(block, mode)[lane] == value


def test_code1_cuda_rule_all_lanes_and_code3_rule_closed_form():
    # CUDA rule: an out-of-range source returns the caller's own value, so
    # every lane of warp 0 doubles five times: 32.  Code 3's CPU translation
    # skips the add instead, so lane l sums lanes l..31: 32 - l.
    v = o.code1(64, 0)
    assert (v[:32] == 32).all() and (v[32:] == 1).all()
    w = o.code1(64, 1)
    assert (w[:32] == 32 - np.arange(32)).all() and (w[32:] == 1).all()


def test_code4_golden_vote_all_is_zero():
    for block, value in _golden("code4_vote_all.txt"):
        assert (o.code4(block) == value).all()


def test_code4_companions_ballot_and_any():
    tx = np.arange(64, dtype=np.int32)
    pred = (tx % 2).astype(np.int32)
    b = o.shfl(o.BALLOT, o.I32, 32, 64, pred)
    assert (b == 0xAAAAAAAA).all()
    assert (o.shfl(o.ANY, o.I32, 32, 64, pred) == 1).all()
    assert (o.shfl(o.ALL, o.I32, 32, 64, pred) == 0).all()


def test_consecutive_votes_are_independent():
    # Section 3.2 / Code 5: two votes in a row through one exchange array.
    r = o.vote_pair(64)
    assert (r[:, 0] == 0).all() and (r[:, 1] == 1).all()


def test_planted_mistake_without_warp_barriers_fails_the_pins():
    o.debug_fuse_phases(True)
    try:
        bad1 = o.code1(64, 0)
        bad2 = o.vote_pair(64)
    finally:
        o.debug_fuse_phases(False)
    assert bad1[0] != 32 or not (bad1[:32] == 32).all()
    assert not (bad2[:, 1] == 1).all()
    assert o.code1(64, 0)[0] == 32  # switch really restored


# ----------------------------------------------- brute force, warp functions
CASES = [(32, 1), (32, 31), (64, 33), (64, 100), (128, 200), (128, 257)]


@pytest.mark.parametrize("W", WIDTHS)
@pytest.mark.parametrize("block,n", CASES)
def test_shuffles_match_brute_force(W, block, n):
    x = inputs.bits_u32(n, seed=11 + n)
    xl = [int(v) for v in x]
    for fn, params in ((lanes.SHFL_IDX, [0, 1, W - 1, W, 37, -3]),
                       (lanes.SHFL_UP, [0, 1, 3, W - 1, min(W, 31), 31]),
                       (lanes.SHFL_DOWN, [0, 1, 5, W - 1, min(W, 31), 31]),
                       (lanes.SHFL_XOR, [0, 1, 2, W - 1, min(W, 31), 17, 31])):
        for p in params:
            got = o.shfl(fn, o.U32, W, block, x, p)
            want = np.array(lanes.shfl(fn, xl, W, p), dtype=np.uint32)
            np.testing.assert_array_equal(got, want, err_msg=f"fn={fn} p={p}")


@pytest.mark.parametrize("W", WIDTHS)
@pytest.mark.parametrize("block,n", CASES)
def test_votes_and_match_match_brute_force(W, block, n):
    pred = (inputs.uniform_int32(n, 0, 3, seed=5 + n) == 0).astype(np.int32)
    pl = [int(v) for v in pred]
    np.testing.assert_array_equal(o.shfl(o.BALLOT, o.I32, W, block, pred), lanes.ballot(pl, W))
    np.testing.assert_array_equal(o.shfl(o.ANY, o.I32, W, block, pred), lanes.any_all(pl, W, False))
    np.testing.assert_array_equal(o.shfl(o.ALL, o.I32, W, block, pred), lanes.any_all(pl, W, True))
    keys = inputs.uniform_int32(n, 0, 4, seed=9 + n)
    np.testing.assert_array_equal(o.shfl(o.MATCH_ANY, o.I32, W, block, keys),
                                  lanes.match_any([int(v) for v in keys], W))


def test_float_votes_use_nonzero_value_and_shuffles_move_bits():
    x = np.array([0.0, -0.0, 1.5, np.nan] * 8, dtype=np.float32)
    b = o.shfl(o.BALLOT, o.F32, 32, 32, x)
    assert int(b[0]) == sum(1 << i for i in range(32) if i % 4 >= 2)
    nan = np.array([np.float32("nan")] * 32, dtype=np.float32).view(np.uint32) | np.uint32(0x1234)
    y = o.shfl(o.SHFL_XOR, o.F32, 32, 32, nan.view(np.float32), 1)
    np.testing.assert_array_equal(y.view(np.uint32), nan)


# ------------------------------------------------------------- invariants
@pytest.mark.parametrize("W", WIDTHS)
def test_xor_is_a_permutation_of_each_full_tile(W):
    n = 128 * 3
    x = inputs.bits_u32(n, seed=3)
    for m in range(W):
        y = o.shfl(o.SHFL_XOR, o.U32, W, 128, x, m)
        np.testing.assert_array_equal(np.sort(y.reshape(-1, W), 1), np.sort(x.reshape(-1, W), 1))


@pytest.mark.parametrize("W", WIDTHS)
def test_ballot_popcount_equals_predicate_count(W):
    n = 1000
    pred = (inputs.uniform_int32(n, 0, 1, seed=4) == 1).astype(np.int32)
    b = o.shfl(o.BALLOT, o.I32, W, 256, pred)
    leaders = np.arange(0, n, W)
    pop = sum(bin(int(v)).count("1") for v in b[leaders])
    assert pop == int(pred.sum())


@pytest.mark.parametrize("W", WIDTHS)
def test_match_masks_partition_each_tile(W):
    n = 999
    keys = inputs.zipf_keys(n, seed=8)
    m = o.shfl(o.MATCH_ANY, o.I32, W, 128, keys)
    for t0 in range(0, n, W):
        seg = range(t0, min(n, t0 + W))
        total = 0
        for i in seg:
            assert (int(m[i]) >> (i - t0)) & 1  # own bit
            low = int(m[i]) & -int(m[i])
            if low == 1 << (i - t0):  # i leads its group
                total += bin(int(m[i])).count("1")
        assert total == len(seg)


def test_appendix_a_each_lane_runs_each_statement_once():
    for W, B, n in ((32, 64, 100), (8, 128, 300), (2, 32, 33)):
        c = o.reduce_counts(W, B, n)
        assert (c[0] == 1).all()
        assert (c[1] == int(math.log2(W))).all()
        per_block = c[2].reshape(-1, B)
        assert (per_block[:, :32] == 1).all() and (per_block[:, 32:] == 0).all()


# ---------------------------------------------------------------- reduce
def _np_seg_reduce(op, x, L):
    starts = np.arange(0, x.size, L)
    if op == o.SUM:
        r = np.add.reduceat(x.astype(np.int64), starts)
        return (r & 0xFFFFFFFF).astype(np.uint32).view(x.dtype)
    uf = {o.MIN: np.minimum, o.MAX: np.maximum, o.AND: np.bitwise_and,
          o.OR: np.bitwise_or, o.XOR: np.bitwise_xor}[op]
    return uf.reduceat(x, starts)


@pytest.mark.parametrize("dt", [o.I32, o.U32])
@pytest.mark.parametrize("op", [o.SUM, o.MIN, o.MAX, o.AND, o.OR, o.XOR])
@pytest.mark.parametrize("W", WIDTHS)
def test_int_reduce_emulation_equals_numpy(dt, op, W):
    n, B = 1000, 128
    x = inputs.bits_u32(n, seed=21).view(np.int32 if dt == o.I32 else np.uint32)
    tile, _ = o.reduce_emulate(op, dt, W, B, o.TILE, x)
    np.testing.assert_array_equal(tile, _np_seg_reduce(op, x, W))
    blk, _ = o.reduce_emulate(op, dt, W, B, o.BLOCK, x)
    np.testing.assert_array_equal(blk, _np_seg_reduce(op, x, B))
    for L in (W, B, n):
        bits, _, _ = o.reduce_ref(op, dt, L, x)
        np.testing.assert_array_equal(bits, _np_seg_reduce(op, x, L))


def test_block_sum_of_the_64x256_int32_workload_equals_numpy():
    x = inputs.uniform_int32(16384, -1000, 1000, seed=inputs.BASE_SEED + 0)
    got, _ = o.reduce_emulate(o.SUM, o.I32, 32, 256, o.BLOCK, x)
    np.testing.assert_array_equal(got, x.reshape(64, 256).sum(1).astype(np.int32))


def test_fp32_sum_tree_order_closed_forms():
    # Width-4 tile tree: (x0 + x2) + (x1 + x3).  1e8 + 1 rounds to 1e8 in fp32
    # (spacing 8), so [1e8, -1e8, 1, 1] sums to 0 in the plain tree while the
    # compensated pairs recover the exact 2; [1e8, 1, -1e8, 1] pairs the big
    # terms first and the plain tree is exact too.
    a = np.array([1e8, -1e8, 1, 1], dtype=np.float32)
    b = np.array([1e8, 1, -1e8, 1], dtype=np.float32)
    assert o.reduce_emulate(o.SUM, o.F32, 4, 32, o.TILE, a)[0][0] == 0.0
    assert o.reduce_emulate(o.SUM, o.F32, 4, 32, o.TILE, a, True)[0][0] == 2.0
    assert o.reduce_emulate(o.SUM, o.F32, 4, 32, o.TILE, b)[0][0] == 2.0
    # a left-to-right sum of b would give ((1e8 + 1) - 1e8) + 1 = 1: the
    # emulation really uses the tree order
    assert np.float32(np.float32(np.float32(1e8) + np.float32(1)) - np.float32(1e8)) + np.float32(1) == 1.0


def _illconditioned(n, seed):
    # values +-2^k, k uniform in [-24, 24]: sums cancel and lose low bits in fp32
    r = inputs.rng(seed)
    k = r.integers(-24, 25, size=n)
    s = np.where(r.random(n) < 0.5, -1.0, 1.0)
    return (s * np.ldexp(1.0, k) * (1 + r.random(n))).astype(np.float32)


@pytest.mark.parametrize("W", WIDTHS)
def test_fp32_reference_is_fsum(W):
    x = _illconditioned(700, seed=W)
    _, ref, ab = o.reduce_ref(o.SUM, o.F32, W, x)
    for g in range(ref.size):
        seg = x[g * W:(g + 1) * W].astype(np.float64)
        assert ref[g] == pytest.approx(math.fsum(seg), rel=1e-15, abs=1e-300)
        assert ab[g] == pytest.approx(math.fsum(np.abs(seg)), rel=1e-12)


@pytest.mark.parametrize("W", WIDTHS)
@pytest.mark.parametrize("scope", [o.TILE, o.BLOCK])
def test_compensated_reduce_meets_1e5_and_plain_is_within_tree_bound(W, scope):
    B, n = 256, 256 * 7 + 45
    x = _illconditioned(n, seed=100 + W)
    L = W if scope == o.TILE else B
    _, ref, ab = o.reduce_ref(o.SUM, o.F32, L, x)
    comp, lo = o.reduce_emulate(o.SUM, o.F32, W, B, scope, x, True)
    assert o.rel_err(comp, ref, ab).max() <= 1e-5
    # hi + lo is the compensated pair's s + e, at least as close as hi alone
    assert (np.abs(comp.astype(np.float64) + lo - ref) <= np.abs(comp.astype(np.float64) - ref) + 1e-30).all()
    plain, _ = o.reduce_emulate(o.SUM, o.F32, W, B, scope, x)
    depth = int(math.log2(W)) + (0 if scope == o.TILE else (B // W + 31) // 32 + 5)
    u = 2.0 ** -24
    assert (np.abs(plain.astype(np.float64) - ref) <= depth * u / (1 - depth * u) * ab + 1e-30).all()


def _cancelling(ntiles, W, seed):
    # each tile: W/2 - 1 big values b, their negatives in shuffled order, and
    # two values in [0, 1): the exact sum is O(1) while sum |x| is ~1e7 W, so
    # a plain fp32 tree drops the small terms and the compensated one keeps them
    r = inputs.rng(seed)
    out = np.empty((ntiles, W), np.float32)
    h = W // 2 - 1
    for t in range(ntiles):
        b = r.uniform(1e6, 1e7, size=h).astype(np.float32)
        row = np.concatenate([b, -r.permutation(b), r.random(2).astype(np.float32)])
        out[t] = r.permutation(row)
    return out.ravel()


def test_plain_fp32_fails_where_compensated_passes():
    # the 1e-5 bar can tell the two apart on these inputs
    x = _cancelling(512, 32, seed=7)
    _, ref, ab = o.reduce_ref(o.SUM, o.F32, 32, x)
    plain, _ = o.reduce_emulate(o.SUM, o.F32, 32, 256, o.TILE, x)
    comp, _ = o.reduce_emulate(o.SUM, o.F32, 32, 256, o.TILE, x, True)
    assert o.rel_err(plain, ref, ab).max() > 1e-5
    assert o.rel_err(comp, ref, ab).max() <= 1e-5


def test_fp32_min_max_are_exact():
    x = inputs.normal_f32(3000, seed=2)
    for op, uf in ((o.MIN, np.minimum), (o.MAX, np.maximum)):
        got, _ = o.reduce_emulate(op, o.F32, 16, 128, o.BLOCK, x)
        np.testing.assert_array_equal(got, uf.reduceat(x, np.arange(0, x.size, 128)))


# ------------------------------------------------------------------ scan
def _np_seg_scan(op, x, W):
    out = np.empty_like(x)
    for t0 in range(0, x.size, W):
        seg = x[t0:t0 + W]
        if op == o.SUM:
            out[t0:t0 + W] = (np.cumsum(seg.astype(np.int64)) & 0xFFFFFFFF).astype(np.uint32).view(x.dtype)
        else:
            uf = {o.MIN: np.minimum, o.MAX: np.maximum, o.AND: np.bitwise_and,
                  o.OR: np.bitwise_or, o.XOR: np.bitwise_xor}[op]
            out[t0:t0 + W] = uf.accumulate(seg)
    return out


@pytest.mark.parametrize("dt", [o.I32, o.U32])
@pytest.mark.parametrize("op", [o.SUM, o.MIN, o.MAX, o.AND, o.OR, o.XOR])
@pytest.mark.parametrize("W", WIDTHS)
def test_int_scan_emulation_equals_numpy(dt, op, W):
    n = 777
    x = inputs.bits_u32(n, seed=31).view(np.int32 if dt == o.I32 else np.uint32)
    got = o.scan_emulate(op, dt, W, 128, x)
    np.testing.assert_array_equal(got, _np_seg_scan(op, x, W))
    bits, _, _ = o.scan_ref(op, dt, W, x)
    np.testing.assert_array_equal(bits, _np_seg_scan(op, x, W))


@pytest.mark.parametrize("W", WIDTHS)
def test_scan_last_lane_equals_tile_reduce(W):
    n = 32 * 40
    xi = inputs.bits_u32(n, seed=41).view(np.int32)
    s = o.scan_emulate(o.SUM, o.I32, W, 256, xi)
    r, _ = o.reduce_emulate(o.SUM, o.I32, W, 256, o.TILE, xi)
    np.testing.assert_array_equal(s[W - 1::W], r)
    xf = _illconditioned(n, seed=42)
    _, sref, sab = o.scan_ref(o.SUM, o.F32, W, xf)
    _, rref, rab = o.reduce_ref(o.SUM, o.F32, W, xf)
    np.testing.assert_array_equal(sref[W - 1::W], rref)
    np.testing.assert_array_equal(sab[W - 1::W], rab)


@pytest.mark.parametrize("W", WIDTHS)
def test_fp32_scan_reference_is_fsum_prefix(W):
    x = _illconditioned(300, seed=50 + W)
    _, ref, ab = o.scan_ref(o.SUM, o.F32, W, x)
    for i in range(x.size):
        seg = x[i - i % W:i + 1].astype(np.float64)
        assert ref[i] == pytest.approx(math.fsum(seg), rel=1e-15, abs=1e-300)
        assert ab[i] == pytest.approx(math.fsum(np.abs(seg)), rel=1e-12)


@pytest.mark.parametrize("W", WIDTHS)
def test_compensated_scan_meets_1e5(W):
    x = _illconditioned(4096 + 77, seed=60 + W)
    _, ref, ab = o.scan_ref(o.SUM, o.F32, W, x)
    comp = o.scan_emulate(o.SUM, o.F32, W, 256, x, True)
    assert o.rel_err(comp, ref, ab).max() <= 1e-5
    plain = o.scan_emulate(o.SUM, o.F32, W, 256, x)
    d = int(math.log2(W))
    u = 2.0 ** -24
    assert (np.abs(plain.astype(np.float64) - ref) <= d * u / (1 - d * u) * ab + 1e-30).all()


# ------------------------------------------------------------ compaction
@pytest.mark.parametrize("W", WIDTHS)
@pytest.mark.parametrize("n", [0, 1, 31, 1000, 4096 + 3])
@pytest.mark.parametrize("d", [0.0, 0.1, 0.5, 0.9, 1.0])
def test_compaction_is_the_stable_filter(W, n, d):
    keys = inputs.uniform_u31(n, seed=70 + n)
    t = inputs.density_threshold(d)
    got, cnt = o.ballot_compact(o.I32, W, 128, keys, t)
    want = keys[keys < t]
    assert cnt == want.size
    np.testing.assert_array_equal(got, want)


def test_compaction_count_is_sum_of_ballot_popcounts():
    n = 5000
    keys = inputs.uniform_u31(n, seed=71)
    t = inputs.density_threshold(0.5)
    _, cnt = o.ballot_compact(o.I32, 32, 256, keys, t)
    b = o.shfl(o.BALLOT, o.I32, 32, 256, (keys < t).astype(np.int32))
    assert cnt == sum(bin(int(v)).count("1") for v in b[::32])


def test_compaction_signed_and_unsigned_compare():
    keys = np.array([-5, 3, 2**31 - 1, -2**31, 0], dtype=np.int32)
    got, _ = o.ballot_compact(o.I32, 32, 32, keys, 1)
    np.testing.assert_array_equal(got, [-5, -2**31, 0])
    got, _ = o.ballot_compact(o.U32, 32, 32, keys.view(np.uint32), 2**31)
    np.testing.assert_array_equal(got.view(np.int32), [3, 2**31 - 1, 0])


# ------------------------------------------------------------- histogram
@pytest.mark.parametrize("W", WIDTHS)
@pytest.mark.parametrize("n", [0, 1, 33, 5000])
def test_match_histogram_is_bincount(W, n):
    keys = inputs.zipf_keys(n, seed=80 + n)
    keys[::7] = -3          # outside the bins: ignored
    keys[1::11] = 300
    hist, ign = o.match_histogram(W, 128, keys, 256)
    inside = keys[(keys >= 0) & (keys < 256)]
    np.testing.assert_array_equal(hist, np.bincount(inside, minlength=256))
    assert ign == n - inside.size
    assert int(hist.sum()) + ign == n


def test_zipf_generator_shape():
    keys = inputs.zipf_keys(200000, seed=1)
    p0 = (keys == 0).mean()
    assert abs(p0 - 0.2065) < 0.005 and keys.min() >= 0 and keys.max() < 256


# --------------------------------------------------------------- batched
def test_batch_reference_is_fsum_and_bincount_per_array():
    lens = inputs.loguniform_lengths(40, 32, 4096, seed=90)
    off = np.concatenate([[0], np.cumsum(lens)])
    vals = _illconditioned(int(off[-1]), seed=91)
    keys = inputs.zipf_keys(int(off[-1]), seed=92)
    sums, ab, hists = o.batch_ref(off, vals, keys)
    for a in range(lens.size):
        seg = vals[off[a]:off[a + 1]].astype(np.float64)
        assert sums[a] == pytest.approx(math.fsum(seg), rel=1e-15, abs=1e-300)
        assert ab[a] == pytest.approx(math.fsum(np.abs(seg)), rel=1e-12)
        np.testing.assert_array_equal(hists[a], np.bincount(keys[off[a]:off[a + 1]], minlength=256))


def test_loguniform_lengths_range():
    lens = inputs.loguniform_lengths(10000, 32, 2**20, seed=93)
    assert lens.min() >= 32 and lens.max() <= 2**20
    assert 0.85e5 < lens.mean() < 1.15e5  # mean of the log-uniform law: (b - a) / ln(b / a) ~ 1.0e5


@pytest.mark.parametrize("L", [100, 4096, 70_001])
def test_long_segment_scan_reference_equals_numpy(L):
    # segments longer than a tile: the reference of block- and grid-scope scans
    x = inputs.bits_u32(70_001, seed=L).view(np.int32)
    bits, _, _ = o.scan_ref(o.SUM, o.I32, L, x)
    np.testing.assert_array_equal(bits, _np_seg_scan(o.SUM, x, L))
    f = inputs.normal_f32(70_001, seed=L + 1)
    _, ref, ab = o.scan_ref(o.SUM, o.F32, L, f)
    for t0 in range(0, f.size, L):
        seg = f[t0:t0 + L].astype(np.float64)
        want = np.cumsum(seg)  # FP64 running sum: close to the exact prefix for these sizes
        assert np.allclose(ref[t0:t0 + L], want, rtol=0, atol=1e-9 * np.abs(seg).sum() + 1e-12)


# ------------------------------------------- grid reduce-then-broadcast pins
def test_grid_sub_min_integers_by_python_ints():
    for dt, lo, hi in ((o.I32, -2**31, 2**31), (o.U32, 0, 2**32)):
        x = inputs.bits_u32(257, seed=3 + dt)
        x = x.view(np.int32) if dt == o.I32 else x
        y = o.grid_sub_min(dt, x)
        m = min(int(v) for v in x)
        want = [((int(v) - m) % 2**32) for v in x]
        assert [int(v) % 2**32 for v in y] == want
        assert int(y[int(np.argmin(x))]) == 0  # the minimum's lane gets 0
    # a constant array maps to zeros; the wrap of the extremes
    assert (o.grid_sub_min(o.I32, np.full(9, -7, np.int32)) == 0).all()
    np.testing.assert_array_equal(o.grid_sub_min(o.I32, np.array([2**31 - 1, -2**31], np.int32)),
                                  np.array([-1, 0], np.int32))


def test_grid_sub_min_fp32_is_one_correct_rounding():
    from fractions import Fraction
    x = inputs.normal_f32(513, seed=8) * np.float32(1e3)
    x[7] = np.float32(-0.0)
    y = o.grid_sub_min(o.F32, x)
    m = Fraction(float(x.min()))
    for v, got in zip(x, y):
        exact = Fraction(float(v)) - m
        # the fp32 value nearest the exact difference (ties away from an odd last bit)
        f = np.float32(float(exact))
        if Fraction(float(f)) != exact:
            lo, hi = sorted((f, np.nextafter(f, np.float32(np.inf) if Fraction(float(f)) < exact else
                                             np.float32(-np.inf))), key=float)
            dlo, dhi = exact - Fraction(float(lo)), Fraction(float(hi)) - exact
            f = lo if dlo < dhi or (dlo == dhi and (int(lo.view(np.uint32)) & 1) == 0) else hi
        assert float(got) == float(f)
    assert (y >= 0).all() and y[int(np.argmin(x))] == 0


def test_grid_normalize_closed_forms():
    ref, norm = o.grid_normalize_ref(np.array([3, 4], np.float32))
    assert norm == 5.0 and list(ref) == [0.6, 0.8]
    for n in (1, 16, 1000):
        ref, norm = o.grid_normalize_ref(np.full(n, 2.5, np.float32))
        assert norm == pytest.approx(2.5 * math.sqrt(n), rel=1e-15)
        assert np.allclose(ref, 1 / math.sqrt(n), rtol=1e-15)
    x = inputs.normal_f32(4097, seed=9)
    ref, norm = o.grid_normalize_ref(x)
    assert math.fsum((ref * ref).tolist()) == pytest.approx(1.0, rel=1e-14)
    assert np.all(np.sign(ref) == np.sign(x))
    ref2, norm2 = o.grid_normalize_ref(x * np.float32(2.0 ** 20))  # power-of-two scaling is exact
    np.testing.assert_array_equal(ref2, ref)
    assert norm2 == norm * 2.0 ** 20
    perm = np.random.default_rng(1).permutation(x.size)
    ref3, _ = o.grid_normalize_ref(x[perm])
    np.testing.assert_array_equal(ref3, ref[perm])


def test_fp32_min_total_order_by_python_sort_key():
    rng = np.random.default_rng(5)
    pool = np.array([0.0, -0.0, 1.5, -1.5, np.inf, -np.inf, np.nan, 3e-45, -3e-45, 1e38], np.float32)
    for _ in range(200):
        a = rng.choice(pool, size=int(rng.integers(1, 8)))
        nums = [float(v) for v in a if not math.isnan(float(v))]
        m = o.fp32_min_total_order(a)
        if not nums:
            assert math.isnan(float(m))
            continue
        want = min(nums, key=lambda v: (v, 0 if math.copysign(1.0, v) < 0 else 1))
        assert float(m) == want and math.copysign(1.0, float(m)) == math.copysign(1.0, want)


# ------------------------------------------------ coalesced-group pins
def _per_warp_compacted(x, act):
    """numpy form: each warp's active values, in lane order, via boolean masks."""
    nw = (x.size + 31) // 32
    for w in range(nw):
        sl = slice(32 * w, min(32 * (w + 1), x.size))
        a = act[sl] != 0
        yield sl, np.flatnonzero(a), x[sl][a]


@pytest.mark.parametrize("density", [0.0, 0.3, 0.9, 1.0])
def test_coalesced_matches_numpy_compaction(density):
    n = 32 * 40 + 13
    x = inputs.bits_u32(n, seed=21).view(np.int32)
    act = (inputs.uniform_u31(n, seed=22) < inputs.density_threshold(density)).astype(np.int32) if density < 1 else \
        np.ones(n, np.int32)
    outs = {fn: o.coalesced(fn, o.I32, 128, x, act, 3) for fn in range(10)}
    for sl, lanes_, vals in _per_warp_compacted(x, act):
        size = vals.size
        for r, lane in enumerate(lanes_):
            i = sl.start + lane
            got = {fn: int(outs[fn][0][i]) for fn in outs}
            assert all(outs[fn][1][i] for fn in outs)
            assert got[o.CG_SIZE] == size and got[o.CG_RANK] == r
            assert got[o.CG_SHFL] == int(vals[3 % size].view(np.uint32))
            assert got[o.CG_SHFL_UP] == int((vals[r - 3] if r >= 3 else vals[r]).view(np.uint32))
            assert got[o.CG_SHFL_DOWN] == int((vals[r + 3] if r + 3 < size else vals[r]).view(np.uint32))
            preds = vals != 0
            assert got[o.CG_BALLOT] == int(sum(1 << k for k in range(size) if preds[k]))
            assert got[o.CG_ANY] == int(preds.any()) and got[o.CG_ALL] == int(preds.all())
            assert got[o.CG_REDUCE_SUM] == int(vals.astype(np.int64).sum()) % 2**32
            assert got[o.CG_SCAN_SUM] == int(np.cumsum(vals.astype(np.int64))[r]) % 2**32
        inactive = np.setdiff1d(np.arange(sl.stop - sl.start), lanes_) + sl.start
        assert not outs[o.CG_SIZE][1][inactive].any()


def test_coalesced_full_warp_is_the_warp_function():
    # every lane active: the coalesced group is the warp, so its functions are
    # the width-32 warp functions already pinned (shfl, ballot, tile reduce/scan)
    n = 32 * 16
    x = inputs.bits_u32(n, seed=23).view(np.int32)
    act = np.ones(n, np.int32)
    for fn, ref in ((o.CG_SHFL, o.shfl(o.SHFL_IDX, o.I32, 32, 256, x, 5)),
                    (o.CG_SHFL_UP, o.shfl(o.SHFL_UP, o.I32, 32, 256, x, 5)),
                    (o.CG_SHFL_DOWN, o.shfl(o.SHFL_DOWN, o.I32, 32, 256, x, 5)),
                    (o.CG_BALLOT, o.shfl(o.BALLOT, o.I32, 32, 256, x, 0))):
        np.testing.assert_array_equal(o.coalesced(fn, o.I32, 256, x, act, 5)[0], ref.view(np.uint32))
    sums, _, _ = o.reduce_ref(o.SUM, o.I32, 32, x)
    np.testing.assert_array_equal(o.coalesced(o.CG_REDUCE_SUM, o.I32, 256, x, act)[0].view(np.int32),
                                  np.repeat(sums.view(np.int32), 32))
    np.testing.assert_array_equal(o.coalesced(o.CG_SCAN_SUM, o.I32, 256, x, act)[0],
                                  o.scan_emulate(o.SUM, o.I32, 32, 256, x).view(np.uint32))


def test_filter_multiset_equals_sorted_stable_compaction():
    keys = inputs.uniform_u31(20_000, seed=24).view(np.int32)
    for d in (0.0, 0.25, 1.0):
        t = inputs.density_threshold(d)
        kept, cnt = o.filter_multiset(o.I32, keys, t)
        stable, scnt = o.ballot_compact(o.I32, 32, 256, keys, t)
        assert cnt == scnt
        np.testing.assert_array_equal(kept, np.sort(stable.astype(np.int64)))


# ------------------------------------- vote statistics / integral image pins
@pytest.mark.parametrize("W", WIDTHS)
def test_vote_stats_by_ballots_of_the_pinned_vote_oracle(W):
    # tile any/all/popcount from the oracle's own pinned ballots (bit r of the
    # tile-local mask = rank r's predicate), summed per segment by Python loops
    n, seg = 32 * 37 + 5, 32 * 8
    pred = (inputs.uniform_u31(n, seed=W) < inputs.density_threshold(0.9)).astype(np.int32)
    pred[::97] = 0
    st = o.vote_stats(W, pred, seg)
    ball = o.shfl(o.BALLOT, o.I32, W, 256, pred)
    for s in range(st.shape[0]):
        a = al = pc = 0
        for t0 in range(s * seg, min(n, (s + 1) * seg), W):
            m = int(ball[t0])
            full = (1 << W) - 1
            a += m != 0
            al += m == full
            pc += bin(m).count("1")
        assert list(st[s]) == [a, al, pc]


def test_vote_stats_closed_forms():
    assert list(o.vote_stats(32, np.ones(64, np.int32), 64)[0]) == [2, 2, 64]
    assert list(o.vote_stats(8, np.zeros(40, np.int32), 40)[0]) == [0, 0, 0]
    # ragged: 3 lanes of a 4-wide tile, all true -> any but not all (padding is false)
    assert list(o.vote_stats(4, np.ones(7, np.int32), 8)[0]) == [2, 1, 7]


def test_integral_image_brute_force_and_closed_forms():
    img = (inputs.bits_u32(2 * 5 * 7, seed=30) & 0xFF).astype(np.uint8).reshape(2, 5, 7)
    got = o.integral_image(img)
    for b in range(2):
        for y in range(5):
            for x in range(7):
                assert int(got[b, y, x]) == int(img[b, :y + 1, :x + 1].astype(np.int64).sum())
    ones = np.ones((1, 9, 13), np.uint8)
    yy, xx = np.mgrid[0:9, 0:13]
    np.testing.assert_array_equal(o.integral_image(ones)[0], ((yy + 1) * (xx + 1)).astype(np.uint32))
    # the recurrence I = img + I(up) + I(left) - I(up-left), mod 2^32, on 32-bit pixels
    big = inputs.bits_u32(3 * 11 * 17, seed=31).reshape(3, 11, 17)
    I = o.integral_image(big).astype(np.int64)
    im = big.astype(np.int64)
    rec = im[:, 1:, 1:] + I[:, :-1, 1:] + I[:, 1:, :-1] - I[:, :-1, :-1]
    np.testing.assert_array_equal(rec % 2**32, I[:, 1:, 1:])
