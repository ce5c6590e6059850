"""GPU parity: every op through the C ABI against the CPU oracle.

Integer, vote, match, compaction and histogram results must be bit-exact.
Every fp32 sum and scan is checked against the FP64 definition (the
oracle's reference value r and sum|x| of the same inputs): compensated
results to |y - r| / max(|r|, 2^-24 sum|x|) <= 1e-5 at every output, plain
ones to the tree-depth bound gamma_h sum|x| of the order the kernel states
(tests/fpcheck.py); fp32 min/max are exact.  fp32 TILE/BLOCK reductions and
tile scans follow the oracle's association order exactly, so they must also
be bit-exact against its fp32 emulation -- a second layer on top of the
definition.  Outputs are poisoned first so that writes past the valid range
are caught.
"""
import numpy as np
import pytest

import oracle as o
from paper_2112_10034_gb300 import inputs
from tests import fpcheck as fc

pytestmark = pytest.mark.gpu

WIDTHS = [2, 4, 8, 16, 32]
POISON = 0x7FBADBAD
TOL = 1e-5


@pytest.fixture(scope="module")
def cox():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_10034_gb300 import build, cox as c
    build.build()
    c.lib()
    return c


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def poisoned(n, dtype, extra=64):
    import torch
    t = torch.full((n + extra,), POISON, dtype=torch.int32, device="cuda")
    return t.view(dtype) if dtype != torch.int32 else t


def host(t):
    return t.cpu().numpy()


def _np_dtype(dt):
    return {o.I32: np.int32, o.U32: np.uint32, o.F32: np.float32}[dt]


def _data(dt, n, seed):
    if dt == o.F32:
        return inputs.normal_f32(n, seed)
    return inputs.bits_u32(n, seed).view(_np_dtype(dt))


def _check_reduce_def(got, op, dt, W, B, scope, x, comp=False, what=""):
    """TILE/BLOCK reduction results against the plain definition."""
    seg = W if scope == o.TILE else B
    bits, ref, ab = o.reduce_ref(op, dt, seg, x)
    if dt == o.F32 and op == o.SUM:
        depth = fc.tile_depth(W) if scope == o.TILE else fc.block_depth(W, B)
        fc.assert_fp64(got.view(np.float32), ref, ab, comp, depth, what)
    else:
        np.testing.assert_array_equal(got.view(np.uint32), bits.view(np.uint32), err_msg=what)


def _check_scan_def(got, op, dt, W, x, comp=False, what=""):
    """Tile-scan results against the plain definition."""
    bits, ref, ab = o.scan_ref(op, dt, W, x)
    if dt == o.F32 and op == o.SUM:
        return fc.assert_fp64(got.view(np.float32), ref, ab, comp, fc.tile_depth(W), what)
    np.testing.assert_array_equal(got.view(np.uint32), bits.view(np.uint32), err_msg=what)


def _torch_view(t, dt):
    import torch
    return t.view(torch.float32) if dt == o.F32 else t.view(torch.int32)


# ---------------------------------------------------------------- cox_shfl
@pytest.mark.parametrize("W", WIDTHS)
@pytest.mark.parametrize("n", [1, 255, 256 * 8 + 77, 100_003])
def test_shfl_all_functions(cox, W, n):
    import torch
    x = inputs.bits_u32(n, seed=n + W)
    xi = x.view(np.int32)
    xd = dev(xi)
    for fn, params in ((o.SHFL_IDX, [0, 3, -1]), (o.SHFL_UP, [0, 1, W - 1, 31]),
                       (o.SHFL_DOWN, [1, W // 2, 31]), (o.SHFL_XOR, [1, W - 1, 17])):
        for p in params:
            out = poisoned(n, torch.int32)
            assert cox.cox_shfl(fn, cox.COX_U32, W, 256, xd.data_ptr(), out.data_ptr(), n, p, cox.FULL_MASK,
                                None) == 0
            got = host(out)
            np.testing.assert_array_equal(got[:n].view(np.uint32), o.shfl(fn, o.U32, W, 256, x, p))
            assert (got[n:] == POISON).all()
    pred = (inputs.uniform_int32(n, 0, 2, seed=n) == 0).astype(np.int32)
    keys = inputs.uniform_int32(n, 0, 3, seed=n + 1)
    for fn, arr in ((o.BALLOT, pred), (o.ANY, pred), (o.ALL, pred), (o.MATCH_ANY, keys)):
        out = poisoned(n, torch.int32)
        assert cox.cox_shfl(fn, cox.COX_I32, W, 128, dev(arr).data_ptr(), out.data_ptr(), n, 0, cox.FULL_MASK,
                            None) == 0
        got = host(out)
        np.testing.assert_array_equal(got[:n].view(np.uint32), o.shfl(fn, o.I32, W, 128, arr).view(np.uint32))
        assert (got[n:] == POISON).all()


def test_shfl_float_votes_and_unaligned_pointer(cox):
    import torch
    f = inputs.normal_f32(5000, seed=3)
    f[::3] = 0.0
    f[1::7] = -0.0
    for fn in (o.BALLOT, o.ANY, o.ALL):
        got = host(cox.shfl(fn, dev(f), width=8))
        np.testing.assert_array_equal(got.view(np.uint32), o.shfl(fn, o.F32, 8, 256, f).view(np.uint32))
    # a view that starts 4 bytes past a 16-byte boundary takes the scalar path
    x = inputs.bits_u32(4097, seed=4).view(np.int32)
    full = dev(x)
    view = full[1:]
    out = torch.empty(4096, dtype=torch.int32, device="cuda")
    assert cox.cox_shfl(o.SHFL_XOR, cox.COX_I32, 16, 256, view.data_ptr(), out.data_ptr(), 4096, 5,
                        cox.FULL_MASK, None) == 0
    np.testing.assert_array_equal(host(out), o.shfl(o.SHFL_XOR, o.I32, 16, 256, x[1:], 5))


def test_code1_and_code4_on_the_gpu(cox):
    # Code 1: all-ones, shfl_down offsets 16..1 accumulate 32 into lane 0
    # (every lane under the CUDA rule); Code 4: all(tx % 2) is 0 everywhere.
    import torch
    ones = torch.ones(64, dtype=torch.int32, device="cuda")
    v = ones.clone()
    for off in (16, 8, 4, 2, 1):
        v = v + cox.shfl(o.SHFL_DOWN, v, width=32, block_dim=64, param=off)
    got = host(v)
    # the oracle's Code 1 runs the loop in warp 0 only; here every warp runs it
    np.testing.assert_array_equal(got[:32], o.code1(64, 0)[:32])
    assert (got == 32).all()
    tx = torch.arange(64, dtype=torch.int32, device="cuda") % 2
    assert (host(cox.shfl(o.ALL, tx, width=32, block_dim=64)) == 0).all()
    assert (host(cox.shfl(o.BALLOT, tx, width=32, block_dim=64)).view(np.uint32) == 0xAAAAAAAA).all()


# --------------------------------------------------------- cox_tile_reduce
OPS = [(o.I32, o.SUM), (o.I32, o.MIN), (o.I32, o.MAX), (o.I32, o.AND), (o.I32, o.OR), (o.I32, o.XOR),
       (o.U32, o.MIN), (o.U32, o.MAX), (o.F32, o.SUM), (o.F32, o.MIN), (o.F32, o.MAX)]


@pytest.mark.parametrize("dt,op", OPS)
@pytest.mark.parametrize("W", WIDTHS)
def test_tile_and_block_reduce_match_the_emulation(cox, dt, op, W):
    import torch
    for n, B in ((1, 32), (1000, 96), (256 * 40 + 13, 256), (5000, 1024)):
        x = _data(dt, n, seed=n + op + 10 * W)
        xd = dev(x.view(np.int32))
        for scope in (o.TILE, o.BLOCK):
            m = o.n_out(scope, n, W, B)
            out = poisoned(m, torch.int32)
            assert cox.cox_tile_reduce(op, dt, W, B, scope, xd.data_ptr(), out.data_ptr(), n, 0, None, None, 0,
                                       None) == 0
            got = host(out)
            want, _ = o.reduce_emulate(op, dt, W, B, scope, x)
            np.testing.assert_array_equal(got[:m].view(np.uint32), want.view(np.uint32),
                                          err_msg=f"n={n} B={B} scope={scope}")
            _check_reduce_def(got[:m], op, dt, W, B, scope, x, what=f"n={n} B={B} scope={scope}")
            assert (got[m:] == POISON).all()


@pytest.mark.parametrize("W", WIDTHS)
@pytest.mark.parametrize("B", [32, 96, 256, 1024])
def test_block_reduce_persistent_path_and_compensation(cox, W, B):
    # enough logical blocks for the persistent warp kernel (more than 4 per SM)
    import torch
    n = B * 1500 + 7
    x = inputs.normal_f32(n, seed=B + W)
    xd = dev(x)
    for comp in (False, True):
        m = o.n_out(o.BLOCK, n, W, B)
        out = torch.empty(m, dtype=torch.float32, device="cuda")
        lo = torch.empty(m, dtype=torch.float32, device="cuda")
        assert cox.cox_tile_reduce(o.SUM, o.F32, W, B, o.BLOCK, xd.data_ptr(), out.data_ptr(), n,
                                   1 if comp else 0, lo.data_ptr(), None, 0, None) == 0
        want, wlo = o.reduce_emulate(o.SUM, o.F32, W, B, o.BLOCK, x, comp)
        np.testing.assert_array_equal(host(out), want)
        _check_reduce_def(host(out), o.SUM, o.F32, W, B, o.BLOCK, x, comp)
        if comp:
            np.testing.assert_array_equal(host(lo), wlo)
    xi = inputs.bits_u32(n, seed=5).view(np.int32)
    got = host(cox.tile_reduce(dev(xi), o.SUM, W, B, o.BLOCK))
    np.testing.assert_array_equal(got, o.reduce_ref(o.SUM, o.I32, B, xi)[0])


@pytest.mark.parametrize("W", WIDTHS)
def test_tile_reduce_compensated_low_word(cox, W):
    n = 32 * 1000 + 5
    x = inputs.normal_f32(n, seed=W)
    out, lo = cox.tile_reduce(dev(x), o.SUM, W, 256, o.TILE, compensated=True, with_lo=True)
    want, wlo = o.reduce_emulate(o.SUM, o.F32, W, 256, o.TILE, x, True)
    np.testing.assert_array_equal(host(out), want)
    np.testing.assert_array_equal(host(lo), wlo)
    _check_reduce_def(host(out), o.SUM, o.F32, W, 256, o.TILE, x, comp=True)
    # out + lo is the compensated pair's exact sum s + e: closer still to r
    _, ref, ab = o.reduce_ref(o.SUM, o.F32, W, x)
    pair = host(out).astype(np.float64) + host(lo).astype(np.float64)
    assert o.rel_err(pair, ref, ab).max() <= fc.TOL


@pytest.mark.parametrize("W", WIDTHS)
@pytest.mark.parametrize("comp", [False, True])
def test_tile_reduce_row_path_sizes_and_alignment(cox, W, comp):
    """Aligned inputs of >= 32 elements take the row-per-lane TMA kernel (whole
    rows, partial chunks, a partial last row, several chunks per warp);
    inputs offset by 4 bytes take the shuffle kernel.  Sums and low words
    are the emulation's bits; nothing is written past the last tile."""
    import torch
    flags = cox.COX_F_COMPENSATED if comp else 0
    for n in (32, 33, 1024 + 31, 32 * 45 + 7, 2432 * 1024 * 3 + 32 * 5 + 9):
        x = inputs.normal_f32(n, seed=n + 5 * W + comp)
        m = o.n_out(o.TILE, n, W, 256)
        want, wlo = o.reduce_emulate(o.SUM, o.F32, W, 256, o.TILE, x, comp)
        for off in (0, 1):
            xd = torch.zeros(n + 8, dtype=torch.float32, device="cuda")
            xd[off:off + n] = dev(x)
            out = poisoned(m, torch.int32)
            lo = poisoned(m, torch.int32)
            assert cox.cox_tile_reduce(o.SUM, o.F32, W, 256, o.TILE, xd.data_ptr() + 4 * off, out.data_ptr(), n,
                                       flags, lo.data_ptr() if comp else None, None, 0, None) == 0
            got = host(out)
            np.testing.assert_array_equal(got[:m].view(np.uint32), want.view(np.uint32))
            _check_reduce_def(got[:m], o.SUM, o.F32, W, 256, o.TILE, x, comp, what=f"n={n} off={off}")
            assert (got[m:] == POISON).all()
            if comp:
                np.testing.assert_array_equal(host(lo)[:m].view(np.uint32), wlo.view(np.uint32))
    assert cox.device_status() == cox.COX_OK


@pytest.mark.parametrize("W", [2, 8, 32])
@pytest.mark.parametrize("B", [32, 64, 256, 1024])
def test_block_reduce_row_path_tails_and_alignment(cox, W, B):
    """Power-of-two blocks over aligned inputs take the row-per-lane kernel:
    a last block made of full rows, a last block reaching into a partial row,
    a last block shorter than one row, and inputs offset by 4 bytes (the
    shuffle kernel).  Sums, low words and integer sums match the emulation."""
    import torch
    nblk = 4 * 152 + 5  # past the one-CTA-per-block path
    for n in (nblk * B, nblk * B - 32, nblk * B - 19, (nblk - 1) * B + 7):
        x = inputs.normal_f32(n, seed=n + W + B)
        m = o.n_out(o.BLOCK, n, W, B)
        want, wlo = o.reduce_emulate(o.SUM, o.F32, W, B, o.BLOCK, x, True)
        for off in (0, 1):
            xd = torch.zeros(n + 8, dtype=torch.float32, device="cuda")
            xd[off:off + n] = dev(x)
            out = poisoned(m, torch.int32)
            lo = poisoned(m, torch.int32)
            assert cox.cox_tile_reduce(o.SUM, o.F32, W, B, o.BLOCK, xd.data_ptr() + 4 * off, out.data_ptr(), n,
                                       cox.COX_F_COMPENSATED, lo.data_ptr(), None, 0, None) == 0
            got = host(out)
            np.testing.assert_array_equal(got[:m].view(np.uint32), want.view(np.uint32), err_msg=f"n={n} off={off}")
            _check_reduce_def(got[:m], o.SUM, o.F32, W, B, o.BLOCK, x, True, what=f"n={n} off={off}")
            assert (got[m:] == POISON).all()
            np.testing.assert_array_equal(host(lo)[:m].view(np.uint32), wlo.view(np.uint32))
        xi = inputs.bits_u32(n, seed=n).view(np.int32)
        for op in (o.SUM, o.MIN, o.XOR):
            got = host(cox.tile_reduce(dev(xi), op, W, B, o.BLOCK))
            np.testing.assert_array_equal(got, o.reduce_emulate(op, o.I32, W, B, o.BLOCK, xi)[0])
            _check_reduce_def(got, op, o.I32, W, B, o.BLOCK, xi)
    assert cox.device_status() == cox.COX_OK


@pytest.mark.parametrize("W", [2, 32])
def test_tile_reduce_2p26_fp32_full_size(cox, W):
    n = 1 << 26
    x = inputs.normal_f32(n, seed=inputs.BASE_SEED + 2)
    xd = dev(x)
    for comp in (False, True):
        got = cox.tile_reduce(xd, o.SUM, W, 256, o.TILE, compensated=comp, with_lo=comp)
        out, lo = got if comp else (got, None)
        want, wlo = o.reduce_emulate(o.SUM, o.F32, W, 256, o.TILE, x, comp)
        np.testing.assert_array_equal(host(out), want)
        _check_reduce_def(host(out), o.SUM, o.F32, W, 256, o.TILE, x, comp, what="TILE 2^26")
        if comp:
            np.testing.assert_array_equal(host(lo), wlo)
        bo = cox.tile_reduce(xd, o.SUM, W, 256, o.BLOCK, compensated=comp)
        np.testing.assert_array_equal(host(bo), o.reduce_emulate(o.SUM, o.F32, W, 256, o.BLOCK, x, comp)[0])
        _check_reduce_def(host(bo), o.SUM, o.F32, W, 256, o.BLOCK, x, comp, what="BLOCK 2^26")


@pytest.mark.parametrize("dt,op", OPS)
def test_grid_reduce(cox, dt, op):
    for n in (0, 1, 1000, 3_000_001):
        x = _data(dt, n, seed=n + 3)
        got = host(cox.tile_reduce(dev(x.view(np.int32)).view(_torch_dtype(dt)), op, 32, 256, o.GRID,
                                   unsigned=dt == o.U32))
        if n == 0:
            continue
        bits, ref, ab = o.reduce_ref(op, dt, n, x)
        if dt == o.F32 and op == o.SUM:
            for fp64 in (False, True):
                y = host(cox.tile_reduce(dev(x), op, 32, 256, o.GRID, compensated=True, fp64_combine=fp64))
                assert o.rel_err(y, ref, ab).max() <= TOL
        else:
            np.testing.assert_array_equal(got.view(np.uint32), bits.view(np.uint32))


def _torch_dtype(dt):
    import torch
    return torch.float32 if dt == o.F32 else torch.int32


# ----------------------------------------------------------- cox_tile_scan
@pytest.mark.parametrize("dt,op", OPS)
@pytest.mark.parametrize("W", WIDTHS)
def test_tile_scan_matches_the_emulation(cox, dt, op, W):
    import torch
    for n in (1, 31, 256 * 8 * 3 + 45, 70_001):
        x = _data(dt, n, seed=n + W + op)
        out = poisoned(n, torch.int32)
        assert cox.cox_tile_scan(op, dt, W, 256, dev(x.view(np.int32)).data_ptr(), out.data_ptr(), n, 0,
                                 None) == 0
        got = host(out)
        np.testing.assert_array_equal(got[:n].view(np.uint32), o.scan_emulate(op, dt, W, 256, x).view(np.uint32))
        _check_scan_def(got[:n], op, dt, W, x, what=f"n={n}")
        assert (got[n:] == POISON).all()


@pytest.mark.parametrize("W", WIDTHS)
@pytest.mark.parametrize("comp", [False, True])
def test_tile_scan_row_path_sizes_and_alignment(cox, W, comp):
    """Aligned arrays of >= 32 elements take the row-per-lane TMA kernel: whole
    rows, partial chunks of rows, a partial last row, and three chunks per
    persistent warp (the 2^26 test below cycles each warp's ring many times);
    arrays offset by 4 bytes take the shuffle kernel.  Both give the
    emulation's bits."""
    import torch
    sizes = (32, 33, 1024, 1024 + 31, 32 * 45 + 7, 2432 * 1024 * 3 + 32 * 5 + 9)
    flags = cox.COX_F_COMPENSATED if comp else 0
    for n in sizes:
        x = inputs.normal_f32(n, seed=n + 3 * W + comp)
        for off in (0, 1):
            xd = torch.zeros(n + 8, dtype=torch.float32, device="cuda")
            xd[off:off + n] = dev(x)
            out = poisoned(n + 8, torch.int32)
            assert cox.cox_tile_scan(o.SUM, o.F32, W, 256, xd.data_ptr() + 4 * off, out.data_ptr() + 4 * off, n,
                                     flags, None) == 0
            got = host(out)
            want = o.scan_emulate(o.SUM, o.F32, W, 256, x, comp)
            np.testing.assert_array_equal(got[off:off + n].view(np.uint32), want.view(np.uint32))
            _check_scan_def(got[off:off + n], o.SUM, o.F32, W, x, comp, what=f"n={n} off={off}")
            assert (got[:off] == POISON).all() and (got[off + n:] == POISON).all()
    assert cox.device_status() == cox.COX_OK


@pytest.mark.parametrize("W", WIDTHS)
def test_compensated_scan_bits_and_error(cox, W):
    n = 256 * 8 * 10 + 3
    x = inputs.normal_f32(n, seed=77 + W)
    for B in (64, 256, 1024):
        got = host(cox.tile_scan(dev(x), o.SUM, W, B, compensated=True))
        np.testing.assert_array_equal(got, o.scan_emulate(o.SUM, o.F32, W, B, x, True))
        _check_scan_def(got, o.SUM, o.F32, W, x, True, what=f"B={B}")


# ------------------------------------------------------ cox_ballot_compact
@pytest.mark.parametrize("d", [0.0, 0.1, 0.5, 0.9, 1.0])
@pytest.mark.parametrize("B", [64, 256, 1024])
def test_compaction_is_bit_exact(cox, d, B):
    import torch
    t = inputs.density_threshold(d)
    for n in (1, 4096 + 1, 300_007):
        k = inputs.uniform_u31(n, seed=n + B)
        out = poisoned(n, torch.int32)
        got, cnt = cox.ballot_compact(dev(k), t, block_dim=B, out=out)
        want, wcnt = o.ballot_compact(o.I32, 32, B, k, t)
        c = int(cnt.item())
        assert c == wcnt
        g = host(got)
        np.testing.assert_array_equal(g[:c], want)
        assert (g[c:] == POISON).all()


def test_compaction_unsigned_negative_keys_and_unaligned(cox):
    import torch
    k = inputs.bits_u32(100_001, seed=9).view(np.int32)
    for unsigned, t in ((False, 0), (True, 2**31)):
        got, cnt = cox.ballot_compact(dev(k), t, unsigned=unsigned)
        want, wcnt = o.ballot_compact(o.U32 if unsigned else o.I32, 32, 256, k.view(np.uint32) if unsigned else k, t)
        c = int(cnt.item())
        assert c == wcnt
        np.testing.assert_array_equal(host(got)[:c].view(np.uint32), want.view(np.uint32))
    full = dev(k)
    got, cnt = cox.ballot_compact(full[3:], 0)
    want, wcnt = o.ballot_compact(o.I32, 32, 256, k[3:], 0)
    assert int(cnt.item()) == wcnt
    np.testing.assert_array_equal(host(got)[:wcnt], want)


def test_compaction_lookback_timeout_is_reported(cox):
    # Tile 0's descriptor is withheld in the caller-zeroed workspace (both
    # flag bits set: descriptors only grow, so tile 0's publish cannot clear
    # it): tile 1's look-back must give up after the spin limit, record
    # COX_ETIMEOUT, and every CTA must still finish.
    import torch
    n = 8192 * 8
    k = dev(inputs.uniform_u31(n, seed=1))
    ws_bytes = cox.cox_ballot_compact_workspace(n, 256)
    ws = torch.zeros(ws_bytes // 8, dtype=torch.int64, device="cuda")
    ws[256 // 8] = -(1 << 62)  # 0xC000000000000000: tile 0's descriptor, withheld
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    cox.cox_set_spin_limit(1000)
    try:
        st = cox.cox_ballot_compact(cox.COX_I32, 32, 256, k.data_ptr(), n, 2**30, out.data_ptr(), cnt.data_ptr(),
                                    ws.data_ptr(), ws_bytes, cox.COX_F_WS_READY, None)
        assert st == cox.COX_OK
        assert cox.device_status() == cox.COX_ETIMEOUT
    finally:
        cox.cox_set_spin_limit(0)
    assert cox.device_status() == cox.COX_OK  # the word was cleared
    got, c = cox.ballot_compact(k, 2**30)  # and the library still works
    want, wc = o.ballot_compact(o.I32, 32, 256, host(k), 2**30)
    assert int(c.item()) == wc
    np.testing.assert_array_equal(host(got)[:wc], want)


# ----------------------------------------------------- cox_match_histogram
@pytest.mark.parametrize("W", WIDTHS)
@pytest.mark.parametrize("bins", [1, 256, 1000, 8192])
def test_histogram_is_bit_exact(cox, W, bins):
    for n, B in ((1, 32), (5000, 256), (200_003, 1024)):
        z = inputs.zipf_keys(n, seed=n + W, bins=min(bins, 256))
        z[::13] = -1
        z[5::17] = bins + 3
        want, wign = o.match_histogram(W, B, z, bins)
        for native, direct, ballot in ((False, False, False), (True, False, False), (False, True, False),
                                       (False, False, True)):
            hist, ign = cox.match_histogram(dev(z), bins=bins, width=W, block_dim=B, native_match=native,
                                            direct=direct, ballot_match=ballot)
            np.testing.assert_array_equal(host(hist), want)
            assert int(ign.item()) == wign


def test_histogram_flags(cox):
    import torch
    z = torch.zeros(64, dtype=torch.int32, device="cuda")
    h = torch.zeros(256, dtype=torch.int32, device="cuda")
    for bad in (cox.COX_F_NATIVE_MATCH | cox.COX_F_BALLOT_MATCH, cox.COX_F_DIRECT_ATOMICS | cox.COX_F_BALLOT_MATCH,
                cox.COX_F_COMPENSATED):
        assert cox.cox_match_histogram(0, 32, 256, z.data_ptr(), 64, 256, h.data_ptr(), None, bad,
                                       None) == cox.COX_EINVAL


# ------------------------------------------------------------ full sizes
def test_block_sum_64x256_int32(cox):
    x = inputs.uniform_int32(16384, -1000, 1000, seed=inputs.BASE_SEED)
    got = host(cox.tile_reduce(dev(x), o.SUM, 32, 256, o.BLOCK))
    want, _ = o.reduce_emulate(o.SUM, o.I32, 32, 256, o.BLOCK, x)
    np.testing.assert_array_equal(got, want)
    np.testing.assert_array_equal(got, x.reshape(64, 256).sum(1))


@pytest.mark.parametrize("W", [4, 8, 16, 32])
def test_tile_scan_2p26_fp32_full_size(cox, W):
    n = 1 << 26
    x = inputs.normal_f32(n, seed=inputs.BASE_SEED + 1)
    xd = dev(x)
    for comp in (False, True):
        got = host(cox.tile_scan(xd, o.SUM, W, 256, compensated=comp))
        np.testing.assert_array_equal(got, o.scan_emulate(o.SUM, o.F32, W, 256, x, comp))
        _check_scan_def(got, o.SUM, o.F32, W, x, comp, what=f"W={W} comp={comp}")


@pytest.mark.parametrize("d", [0.1, 0.5, 0.9])
def test_compaction_2p28_full_size(cox, d):
    n = 1 << 28
    k = inputs.uniform_u31(n, seed=inputs.BASE_SEED + 2)
    t = inputs.density_threshold(d)
    got, cnt = cox.ballot_compact(dev(k), t)
    want, wcnt = o.ballot_compact(o.I32, 32, 256, k, t)
    c = int(cnt.item())
    assert c == wcnt
    np.testing.assert_array_equal(host(got[:c]), want)
