"""GPU parity of block- and grid-scope scans (cox_scan) against the oracle.

Integer scans must be bit-exact (inclusive and exclusive); fp32 sums must
meet |y - r| / max(|r|, 2^-24 sum|x|) <= 1e-5 against the FP64 prefix when
compensated; min/max are exact.  Outputs past n must stay untouched.
"""
import numpy as np
import pytest

import oracle as o
from paper_2112_10034_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-5
POISON = 0x7FBADBAD


@pytest.fixture(scope="module")
def cox():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_10034_gb300 import build, cox as c
    build.build()
    c.lib()
    return c


def _ident(op, dt):
    if op in (o.SUM, o.OR, o.XOR):
        return 0
    if op == o.AND:
        return -1 if dt == o.I32 else 0xFFFFFFFF
    if dt == o.F32:
        return np.inf if op == o.MIN else -np.inf
    if dt == o.I32:
        return 2**31 - 1 if op == o.MIN else -2**31
    return 0xFFFFFFFF if op == o.MIN else 0


def _exclusive(incl, L, ident):
    ex = np.empty_like(incl)
    ex[1:] = incl[:-1]
    ex[::L] = ident
    return ex


def _run(cox, x_host, op, dt, scope, B, comp, excl, offset=0):
    import torch
    n = x_host.size
    full = torch.from_numpy(np.concatenate([np.zeros(offset, x_host.dtype), x_host])).cuda()
    x = full[offset:]
    out = torch.full((n + 64,), POISON, dtype=torch.int32, device="cuda")
    ws_b = cox.cox_scan_workspace(scope, n)
    ws = torch.empty(max(ws_b, 16), dtype=torch.uint8, device="cuda")
    st = cox.cox_scan(op, dt, scope, B, x.data_ptr(), out.data_ptr(), n, 1 if comp else 0, 1 if excl else 0,
                      ws.data_ptr(), ws_b, None)
    assert st == cox.COX_OK
    g = out.cpu().numpy()
    assert (g[n:] == POISON).all()
    return g[:n]


INT_OPS = [(o.I32, o.SUM), (o.I32, o.MIN), (o.I32, o.MAX), (o.I32, o.XOR), (o.I32, o.AND), (o.U32, o.MIN),
           (o.U32, o.MAX), (o.I32, o.OR)]


@pytest.mark.parametrize("dt,op", INT_OPS)
@pytest.mark.parametrize("n", [1, 1000, 16384, 16385, 3 * 16384 + 7, (1 << 21) + 3])
def test_grid_scan_integers_exact(cox, dt, op, n):
    x = inputs.bits_u32(n, seed=n + op).view(np.int32 if dt == o.I32 else np.uint32)
    want, _, _ = o.scan_ref(op, dt, n, x)
    for excl in (False, True):
        got = _run(cox, x, op, dt, o.GRID, 256, False, excl).view(x.dtype)
        w = _exclusive(want, n, _ident(op, dt)) if excl else want
        np.testing.assert_array_equal(got, w.astype(x.dtype))


def test_grid_scan_unaligned_input_takes_the_plain_load_path(cox):
    n = 5 * 16384 + 11
    x = inputs.bits_u32(n, seed=3).view(np.int32)
    want, _, _ = o.scan_ref(o.SUM, o.I32, n, x)
    got = _run(cox, x, o.SUM, o.I32, o.GRID, 256, False, False, offset=1).view(np.int32)
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("n", [777, 8192, 8193, 5 * 16384 + 3, (1 << 22) + 1])
def test_grid_scan_fp32(cox, n):
    x = inputs.normal_f32(n, seed=n)
    _, ref, ab = o.scan_ref(o.SUM, o.F32, n, x)
    for excl in (False, True):
        got = _run(cox, x, o.SUM, o.F32, o.GRID, 256, True, excl).view(np.float32)
        r, a = (ref, ab) if not excl else (_exclusive(ref, n, 0.0), _exclusive(ab, n, 0.0))
        assert o.rel_err(got, r, a).max() <= TOL
    for op, uf in ((o.MIN, np.minimum), (o.MAX, np.maximum)):
        got = _run(cox, x, op, o.F32, o.GRID, 256, False, False).view(np.float32)
        np.testing.assert_array_equal(got, uf.accumulate(x))


@pytest.mark.parametrize("B", [32, 96, 256, 1024])
def test_block_scan(cox, B):
    n = B * 300 + 17
    xi = inputs.bits_u32(n, seed=B).view(np.int32)
    want, _, _ = o.scan_ref(o.SUM, o.I32, B, xi)
    for excl in (False, True):
        got = _run(cox, xi, o.SUM, o.I32, o.BLOCK, B, False, excl).view(np.int32)
        np.testing.assert_array_equal(got, _exclusive(want, B, 0) if excl else want)
    xf = inputs.normal_f32(n, seed=B + 1)
    _, ref, ab = o.scan_ref(o.SUM, o.F32, B, xf)
    got = _run(cox, xf, o.SUM, o.F32, o.BLOCK, B, True, False).view(np.float32)
    assert o.rel_err(got, ref, ab).max() <= TOL
    got = _run(cox, xf, o.MAX, o.F32, o.BLOCK, B, False, True).view(np.float32)
    ref_max, _, _ = o.scan_ref(o.MAX, o.F32, B, xf)
    np.testing.assert_array_equal(got, _exclusive(ref_max.view(np.float32), B, -np.inf))


def test_scan_argument_checks(cox):
    assert cox.cox_scan(0, 0, 0, 256, 16, 16, 10, 0, 0, None, 0, None) == cox.COX_EINVAL  # TILE scope
    assert cox.cox_scan(0, 0, 2, 256, 16, 16, 10, 0, 2, None, 0, None) == cox.COX_EINVAL  # exclusive = 2
    assert cox.cox_scan(0, 0, 2, 256, 16, 16, 100000, 0, 0, None, 0, None) == cox.COX_ENOMEM
