"""GPU parity of the dynamic-group row: cox_coalesced (warp functions over
coalesced_threads() groups, run by the warp intrinsics with partial member
masks) against the oracle's collapsed-loop executor with active masks, bit
for bit on every active lane, with inactive lanes left untouched; and
cox_filter_aggregated (filter_arr's warp-aggregated atomic), whose output
order depends on the order the atomics land: its count and its kept keys
(as a multiset) must be the oracle's, nothing may be written past the
count, and each coalesced group's keys must sit in one run in lane order.
"""
import numpy as np
import pytest

import oracle as o
from paper_2112_10034_gb300 import inputs

pytestmark = pytest.mark.gpu
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


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


FNS = list(range(10))


@pytest.mark.parametrize("fn", FNS)
@pytest.mark.parametrize("density", [0.0, 0.1, 0.5, 0.97, 1.0])
def test_coalesced_matches_the_oracle(cox, fn, density):
    import torch
    for n in (1, 31, 1000, 70_001):
        act = (inputs.uniform_u31(n, seed=n + fn) < inputs.density_threshold(density)).astype(np.int32) \
            if density < 1 else np.ones(n, np.int32)
        dts = [o.I32] if fn in (o.CG_REDUCE_SUM, o.CG_SCAN_SUM) else [o.I32, o.F32]
        for dt in dts:
            if dt == o.F32:
                x = inputs.normal_f32(n, seed=n + 1)
                x[::5] = 0.0
                x[1::7] = -0.0
            else:
                x = inputs.bits_u32(n, seed=n + 2).view(np.int32)
                x[::3] = 0
            params = [0, 1, 5, 31] if fn in (o.CG_SHFL, o.CG_SHFL_UP, o.CG_SHFL_DOWN) else [0]
            for p in params:
                out = torch.full((n + 16,), POISON, dtype=torch.int32, device="cuda")
                assert cox.cox_coalesced(fn, dt, 128, dev(x.view(np.int32)).data_ptr(), dev(act).data_ptr(),
                                         out.data_ptr(), n, p, None) == 0
                got = out.cpu().numpy().view(np.uint32)
                want, written = o.coalesced(fn, dt, 128, x, act, p)
                np.testing.assert_array_equal(got[:n][written], want[written], err_msg=f"n={n} dt={dt} p={p}")
                assert (got[:n][~written] == POISON).all() and (got[n:] == POISON).all()


def test_coalesced_bad_arguments(cox):
    import torch
    x = torch.zeros(64, dtype=torch.int32, device="cuda")
    assert cox.cox_coalesced(o.CG_SCAN_SUM, o.F32, 128, x.data_ptr(), x.data_ptr(), x.data_ptr(), 64, 0,
                             None) == cox.COX_EINVAL
    assert cox.cox_coalesced(o.CG_SHFL, o.I32, 128, x.data_ptr(), x.data_ptr(), x.data_ptr(), 64, 32,
                             None) == cox.COX_EINVAL
    assert cox.cox_coalesced(o.CG_SIZE, o.I32, 100, x.data_ptr(), x.data_ptr(), x.data_ptr(), 64, 0,
                             None) == cox.COX_EINVAL


@pytest.mark.parametrize("d", [0.0, 0.1, 0.5, 0.9, 1.0])
@pytest.mark.parametrize("n", [1, 1000, 4096, 70_001, 4096 * 37, (1 << 22) + 5])
def test_filter_aggregated(cox, d, n):
    import torch
    # distinct keys (a shuffled range), so every output key names its input slot
    keys = np.random.default_rng(n).permutation(n).astype(np.int32)
    t = int(np.floor(d * n))
    out = torch.full((n + 16,), POISON, dtype=torch.int32, device="cuda")
    cnt = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    assert cox.cox_filter_aggregated(o.I32, dev(keys).data_ptr(), n, t, out.data_ptr(), cnt.data_ptr(),
                                     None) == 0
    got = out.cpu().numpy()
    c = int(cnt.item())
    kept, want_c = o.filter_multiset(o.I32, keys, t)
    assert c == want_c
    np.testing.assert_array_equal(np.sort(got[:c].astype(np.int64)), kept)
    assert (got[c:] == POISON).all()
    # each group (32 consecutive keys of a warp round) occupies one run, in lane order
    slot = np.full(n, -1, np.int64)
    slot[keys] = np.arange(n)
    pos_of_input = np.full(n, -1, np.int64)
    pos_of_input[slot[got[:c]]] = np.arange(c)
    for g0 in range(0, n, 32):
        p = pos_of_input[g0:g0 + 32]
        p = p[p >= 0]
        if p.size:
            assert (np.diff(p) == 1).all()


def test_filter_unsigned_threshold_clamp(cox):
    import torch
    keys = inputs.bits_u32(5000, seed=3)
    for t in (-5, 0, 2**31, 2**32, 2**40):
        out = torch.zeros(5000, dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        assert cox.cox_filter_aggregated(o.U32, dev(keys.view(np.int32)).data_ptr(), 5000, t, out.data_ptr(),
                                         cnt.data_ptr(), None) == 0
        kept, c = o.filter_multiset(o.U32, keys, t)
        assert int(cnt.item()) == c
        np.testing.assert_array_equal(np.sort(out.cpu().numpy()[:c].view(np.uint32).astype(np.int64)), kept)


@pytest.mark.parametrize("n", [4096 * 5, 70_001])
def test_filter_unaligned_keys(cox, n):
    """Keys off the 16-byte grid take plain loads; the result is the same."""
    import torch
    keys = np.random.default_rng(n + 1).permutation(n).astype(np.int32)
    t = n // 3
    d_keys = torch.zeros(n + 4, dtype=torch.int32, device="cuda")
    d_keys[1:n + 1] = dev(keys)
    out = torch.full((n + 16,), POISON, dtype=torch.int32, device="cuda")
    cnt = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    assert cox.cox_filter_aggregated(o.I32, d_keys.data_ptr() + 4, n, t, out.data_ptr(), cnt.data_ptr(), None) == 0
    kept, want_c = o.filter_multiset(o.I32, keys, t)
    c = int(cnt.item())
    assert c == want_c
    got = out.cpu().numpy()
    np.testing.assert_array_equal(np.sort(got[:c].astype(np.int64)), kept)
    assert (got[c:] == POISON).all()
    assert cox.cox_device_status(None) == 0
