"""GPU parity of the batched path (cox_batch_*) against the CPU oracle.

Histograms must be bit-exact; every fp32 sum must meet the 1e-5 bar
|y - r| / max(|r|, 2^-24 sum|x|) against the oracle's FP64 value, and the
double outputs too.  Results must not depend on timing: the same tune gives
the same bits twice, graph replays give the same bits as direct calls.
"""
import ctypes

import numpy as np
import pytest

import oracle as o
from paper_2112_10034_gb300 import inputs

pytestmark = pytest.mark.gpu
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


def make_arrays(lens, seed, misalign=True):
    """Device arrays (values, keys) plus their host concatenation for the oracle.
    Some arrays start 4..12 bytes past a 16-byte boundary (values and keys at the
    same phase, or at different phases) to cover every load path."""
    import torch
    vals, keys, hv, hk = [], [], [], []
    for a, L in enumerate(lens):
        v = inputs.normal_f32(L, seed + 2 * a)
        k = inputs.zipf_keys(L, seed + 2 * a + 1)
        if L > 3 and a % 5 == 0:
            k[::7] = -1     # outside the bins: ignored
            k[1::9] = 256
        pv = (a % 4) if misalign else 0
        pk = pv if a % 3 else (pv + 1) % 4
        bv = torch.empty(L + 4, dtype=torch.float32, device="cuda")
        bk = torch.empty(L + 4, dtype=torch.int32, device="cuda")
        tv, tk = bv[pv:pv + L], bk[pk:pk + L]
        tv.copy_(torch.from_numpy(v))
        tk.copy_(torch.from_numpy(k))
        vals.append(tv)
        keys.append(tk)
        hv.append(v)
        hk.append(k)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    return vals, keys, off, np.concatenate(hv) if hv else np.zeros(0, np.float32), \
        np.concatenate(hk) if hk else np.zeros(0, np.int32)


def check(batch, off, hv, hk, tol=TOL):
    sums, sums64, hists = batch.run()
    ref, ab, want = o.batch_ref(off, hv, hk)
    np.testing.assert_array_equal(hists.cpu().numpy(), want)
    s = sums.cpu().numpy()
    assert o.rel_err(s, ref, ab).max() <= tol
    assert o.rel_err(sums64.cpu().numpy(), ref, ab).max() <= tol
    return s


def test_batch_matches_the_oracle(cox):
    lens = list(inputs.loguniform_lengths(300, 32, 1 << 16, seed=1)) + [0, 1, 2, 3, 5, 7, 0, 33, 0]
    vals, keys, off, hv, hk = make_arrays(lens, seed=100)
    b = cox.Batch(vals, keys)
    check(b, off, hv, hk)


@pytest.mark.parametrize("native", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("width", [2, 8, 32])
@pytest.mark.parametrize("block,cpsm", [(64, 1), (256, 2), (512, 4), (1024, 1), (128, 8)])
def test_every_tune_agrees_and_is_deterministic(cox, width, block, cpsm, native):
    lens = list(inputs.loguniform_lengths(120, 32, 1 << 15, seed=2)) + [0, 4, 9]
    vals, keys, off, hv, hk = make_arrays(lens, seed=200)
    b = cox.Batch(vals, keys, tune=(block, cpsm, width, 8, native))
    first = check(b, off, hv, hk).copy()
    second = b.run()[0].cpu().numpy()
    np.testing.assert_array_equal(first.view(np.uint32), second.view(np.uint32))
    # elements per thread only changes how many loads are in flight: the same bits
    for ept in (4, 16):
        e = cox.Batch(vals, keys, tune=(block, cpsm, width, 8, native, ept))
        np.testing.assert_array_equal(check(e, off, hv, hk).view(np.uint32), first.view(np.uint32))


def test_fp64_combine_for_every_array(cox):
    lens = list(inputs.loguniform_lengths(64, 1 << 12, 1 << 20, seed=3))
    vals, keys, off, hv, hk = make_arrays(lens, seed=300, misalign=False)
    b = cox.Batch(vals, keys, tune=(512, 2, 32, 1, 0))
    check(b, off, hv, hk)
    ref, ab, _ = o.batch_ref(off, hv, hk)
    assert o.rel_err(b.sums64.cpu().numpy(), ref, ab).max() <= 1e-9


def test_graph_replay_equals_direct_call(cox):
    import torch
    lens = list(inputs.loguniform_lengths(200, 32, 1 << 14, seed=4))
    vals, keys, off, hv, hk = make_arrays(lens, seed=400)
    b = cox.Batch(vals, keys)
    direct = [t.clone() for t in b.run()]
    g = b.graph()
    for t in (b.sums, b.sums64, b.hists):
        t.zero_()
    for _ in range(2):
        g.launch(b.stream)
    torch.cuda.synchronize()
    for d, r in zip(direct, (b.sums, b.sums64, b.hists)):
        assert torch.equal(d, r)
    check(b, off, hv, hk)


def test_autotune_picks_a_valid_tune_and_caches_it(cox, tmp_path):
    lens = list(inputs.loguniform_lengths(100, 32, 1 << 14, seed=5))
    vals, keys, off, hv, hk = make_arrays(lens, seed=500)
    b = cox.Batch(vals, keys)
    cache = str(tmp_path / "tune.txt")
    best, ms = b.autotune(reps=1, cache_path=cache)
    assert best.block_dim in (256, 512, 1024) and best.ctas_per_sm in (1, 2, 4) and best.width in (8, 32)
    assert ms > 0
    t = cox.cox_batch_tune()
    assert cox.cox_batch_tune_lookup(cache.encode(), b.A, b.total, ctypes.byref(t)) == cox.COX_OK
    assert t.astuple() == best.astuple()
    assert cox.cox_batch_tune_lookup(cache.encode(), b.A * 64, b.total, ctypes.byref(t)) == cox.COX_EINVAL
    check(b, off, hv, hk)  # runs with the tuned shape


def test_batch_argument_checks(cox):
    import torch
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    lens = np.array([5, 6], dtype=np.int64)
    assert cox.cox_batch_prepare(0, lens.ctypes.data, ws.data_ptr(), 1024, None) == cox.COX_EINVAL
    assert cox.cox_batch_prepare(2, lens.ctypes.data, ws.data_ptr(), 8, None) == cox.COX_ENOMEM
    bad = np.array([5, -1], dtype=np.int64)
    assert cox.cox_batch_prepare(2, bad.ctypes.data, ws.data_ptr(), 1024 * 1024, None) != cox.COX_OK
    t = cox.cox_batch_tune(100, 2, 32, 8, 0)  # block not a multiple of 32
    assert cox.cox_batch_sum_hist(2, 16, 16, ctypes.addressof(t), ws.data_ptr(), 1 << 20, 16, None, 16,
                                  None) == cox.COX_EINVAL
    t = cox.cox_batch_tune(256, 2, 32, 8, 0, 5)  # elements per thread not 4, 8 or 16
    assert cox.cox_batch_sum_hist(2, 16, 16, ctypes.addressof(t), ws.data_ptr(), 1 << 20, 16, None, 16,
                                  None) == cox.COX_EINVAL


def test_batch_full_length_law_sample(cox):
    # 1000 arrays from the batched workload's length law (log-uniform on
    # [32, 2^20]), ~1e8 elements: one tenth of the full 10,000-array batch.
    lens = list(inputs.loguniform_lengths(1000, 32, 1 << 20, seed=inputs.BASE_SEED + 3))
    vals, keys, off, hv, hk = make_arrays(lens, seed=inputs.BASE_SEED + 30, misalign=False)
    b = cox.Batch(vals, keys)
    check(b, off, hv, hk)


def test_per_array_launches_match_the_oracle(cox):
    """cox_batch_percall, the one-launch-per-array baseline, gives the same
    histograms and sums within the tolerance (a different order of additions),
    empty arrays included."""
    import torch
    lens = list(inputs.loguniform_lengths(60, 32, 1 << 16, seed=4)) + [0, 1, 5]
    vals, keys, off, hv, hk = make_arrays(lens, seed=400)
    A = len(lens)
    h_vals = (ctypes.c_void_p * A)(*[v.data_ptr() for v in vals])
    h_keys = (ctypes.c_void_p * A)(*[k.data_ptr() for k in keys])
    h_lens = np.array(lens, dtype=np.int64)
    sums = torch.full((A,), float("nan"), dtype=torch.float32, device="cuda")
    hists = torch.full((A, 256), -1, dtype=torch.int32, device="cuda")
    scr_b = cox.cox_batch_percall_scratch(int(max(lens)))
    scr = torch.empty(scr_b, dtype=torch.uint8, device="cuda")
    assert cox.cox_batch_percall(A, h_vals, h_keys, h_lens.ctypes.data, sums.data_ptr(), hists.data_ptr(),
                                 scr.data_ptr(), scr_b, None, None) == cox.COX_OK
    ref, ab, want = o.batch_ref(off, hv, hk)
    np.testing.assert_array_equal(hists.cpu().numpy(), want)
    assert o.rel_err(sums.cpu().numpy(), ref, ab).max() <= TOL
    assert cox.cox_batch_percall(A, h_vals, h_keys, h_lens.ctypes.data, sums.data_ptr(), hists.data_ptr(),
                                 scr.data_ptr(), 8, None, None) == cox.COX_ENOMEM
