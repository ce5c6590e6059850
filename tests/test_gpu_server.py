"""GPU tests of the request server (cox_server_*).

Each request's result must be the same alone and in a mix with others --
bit for bit, since a request's arithmetic never depends on its batch -- and
must match the oracle: scans and compactions exactly, integer sums exactly,
compensated fp32 sums within 1e-5 (|y - r| / max(|r|, 2^-24 sum|x|)).
Admission must respect the memory budget, and traces must replay both
through the server and with one launch per request.
"""
import numpy as np
import pytest

import oracle as o
from paper_2112_10034_gb300 import inputs
from tests import fpcheck as fc

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


def make_mix(cox, count, seed, lo=1000, hi=1 << 18):
    """Mixed requests: 1/3 reduce (half fp32 compensated, half int32), 1/3
    compensated fp32 scans at widths 4..32, 1/3 int32 compactions at d=0.5."""
    import torch
    sizes = inputs.loguniform_lengths(count, lo, hi, seed)
    kinds = inputs.choice(count, 3, seed + 1)
    reqs = []
    for i, (n, k) in enumerate(zip(sizes, kinds)):
        n = int(n)
        if k == 0:
            if i % 2:
                h = inputs.normal_f32(n, seed + 10 + i)
                r = dict(kind=cox.COX_REQ_REDUCE, compensated=True)
            else:
                h = inputs.uniform_int32(n, -1000, 1000, seed + 10 + i)
                r = dict(kind=cox.COX_REQ_REDUCE)
        elif k == 1:
            h = inputs.normal_f32(n, seed + 10 + i)
            r = dict(kind=cox.COX_REQ_SCAN, compensated=True, width=[4, 8, 16, 32][i % 4])
        else:
            h = inputs.uniform_u31(n, seed + 10 + i)
            r = dict(kind=cox.COX_REQ_COMPACT, threshold=inputs.density_threshold(0.5))
        d = torch.from_numpy(h).cuda()
        req = cox.make_request(r.pop("kind"), d, **r)
        reqs.append((req, d, h))
    return reqs


def check_against_oracle(cox, req, host_in, got):
    g = got.cpu().numpy()
    if req.kind == cox.COX_REQ_SCAN:
        comp = bool(req.flags & 1)
        want = o.scan_emulate(o.SUM, o.F32, req.width, 256, host_in, compensated=comp)
        np.testing.assert_array_equal(g, want)
        _, ref, ab = o.scan_ref(o.SUM, o.F32, req.width, host_in)
        fc.assert_fp64(g, ref, ab, comp, fc.tile_depth(req.width), "served scan")
    elif req.kind == cox.COX_REQ_COMPACT:
        want, cnt = o.ballot_compact(o.I32, 32, 256, host_in, req.threshold)
        assert g.size == cnt
        np.testing.assert_array_equal(g, want)
    elif req.dt == cox.COX_F32:
        _, ref, ab = o.reduce_ref(o.SUM, o.F32, host_in.size, host_in)
        assert o.rel_err(g[:1], ref, ab).max() <= TOL
    else:
        bits, _, _ = o.reduce_ref(o.SUM, o.I32, host_in.size, host_in)
        assert g[0] == bits[0]


def test_each_result_is_the_same_alone_and_in_the_mix(cox):
    mix = make_mix(cox, 45, seed=11)
    srv = cox.Server(1 << 30)
    try:
        tickets = srv.submit_many([r for r, _, _ in mix], keep=[d for _, d, _ in mix])
        for t in tickets:
            srv.wait(t)
        in_mix = [srv.result(t, r) for t, (r, _, _) in zip(tickets, mix)]
        for t in tickets:
            srv.release(t)
        st = srv.stats()
        assert st["completed"] == len(mix) and st["failed"] == 0
        assert st["max_batch"] == len(mix)  # queued together: one launch; each request below runs alone
        for (r, d, h), got in zip(mix, in_mix):
            t = srv.submit(r, keep=d)
            srv.wait(t)
            alone = srv.result(t, r)
            srv.release(t)
            assert alone.shape == got.shape
            assert np.array_equal(alone.cpu().numpy().view(np.uint32), got.cpu().numpy().view(np.uint32))
            check_against_oracle(cox, r, h, got)
        assert srv.stats()["used_bytes"] == 0
    finally:
        srv.close()


def test_full_size_mix_against_the_oracle(cox):
    """Twenty requests of the serving workload's kinds with sizes up to 16M
    elements (several at exactly 2^24, so large requests take many tiles and
    deep look-backs inside one persistent launch), queued together so they
    share launches; every result must match the oracle and the same request
    run alone."""
    count = 20
    mix = make_mix(cox, count, seed=31, lo=1024, hi=1 << 24)
    import torch
    n = 1 << 24  # one request of each kind at the top size
    hs = [inputs.normal_f32(n, 41), inputs.uniform_int32(n, -1000, 1000, 42), inputs.normal_f32(n, 43),
          inputs.uniform_u31(n, 44)]
    kw = [dict(kind=cox.COX_REQ_REDUCE, compensated=True), dict(kind=cox.COX_REQ_REDUCE),
          dict(kind=cox.COX_REQ_SCAN, compensated=True, width=32),
          dict(kind=cox.COX_REQ_COMPACT, threshold=inputs.density_threshold(0.5))]
    for h, r in zip(hs, kw):
        d = torch.from_numpy(h).cuda()
        mix.append((cox.make_request(r.pop("kind"), d, **r), d, h))
    assert max(r.n for r, _, _ in mix) == 1 << 24
    srv = cox.Server(6 << 30)
    try:
        tickets = srv.submit_many([r for r, _, _ in mix], keep=[d for _, d, _ in mix])
        for t in tickets:
            srv.wait(t, timeout_s=120.0)
        in_mix = [srv.result(t, r) for t, (r, _, _) in zip(tickets, mix)]
        for t in tickets:
            srv.release(t)
        st = srv.stats()
        assert st["completed"] == len(mix) and st["failed"] == 0
        assert st["max_batch"] > 1
        for (r, d, h), got in zip(mix, in_mix):
            check_against_oracle(cox, r, h, got)
            t = srv.submit(r, keep=d)
            srv.wait(t, timeout_s=120.0)
            alone = srv.result(t, r)
            srv.release(t)
            assert np.array_equal(alone.cpu().numpy().view(np.uint32), got.cpu().numpy().view(np.uint32))
    finally:
        srv.close()
    assert cox.device_status() == cox.COX_OK


def test_requests_one_at_a_time_match_the_oracle(cox):
    """An idle server launches each request from the submitting thread (a lone
    scan or compaction with the op's own kernel, a lone reduce with one CTA
    per tile in the batch kernel's order); a request must not be marked done
    before its results are in memory, so every result read right after the
    wait must match the oracle."""
    mix = make_mix(cox, 36, seed=51, lo=1000, hi=1 << 20)
    srv = cox.Server(1 << 30)
    try:
        for r, d, h in mix:
            t = srv.submit(r, keep=d)
            srv.wait(t)
            got = srv.result(t, r)
            srv.release(t)
            check_against_oracle(cox, r, h, got)
        st = srv.stats()
        assert st["completed"] == len(mix) and st["failed"] == 0 and st["used_bytes"] == 0
    finally:
        srv.close()
    assert cox.device_status() == cox.COX_OK


def test_admission_respects_the_budget(cox):
    import torch
    budget = 8 << 20
    srv = cox.Server(budget, max_requests=64)
    try:
        x = torch.from_numpy(inputs.normal_f32(300_000, 5)).cuda()  # ~2.4 MB held per scan
        reqs = [cox.make_request(cox.COX_REQ_SCAN, x, width=32, compensated=True) for _ in range(12)]
        tickets = [srv.submit(r) for r in reqs]
        for t in tickets:
            srv.wait(t)
            srv.release(t)
        st = srv.stats()
        assert st["completed"] == 12 and st["peak_bytes"] <= budget and st["batches"] >= 4
        big = torch.empty(3_000_000, dtype=torch.float32, device="cuda")
        with pytest.raises(cox.CoxError) as e:
            srv.submit(cox.make_request(cox.COX_REQ_SCAN, big, width=32))
        assert e.value.status == cox.COX_ENOMEM
    finally:
        srv.close()


def test_trace_replay_server_and_per_call(cox):
    mix = make_mix(cox, 120, seed=21, hi=1 << 16)
    arrivals = inputs.poisson_arrivals(len(mix), 20_000.0, seed=22)
    items = [(float(a), r) for a, (r, _, _) in zip(arrivals, mix)]
    srv = cox.Server(1 << 30)
    try:
        lat, wall = srv.run_trace(items)
        st = srv.stats()
        assert st["completed"] == len(mix) and st["used_bytes"] == 0
        assert min(lat) > 0 and wall >= max(arrivals)
    finally:
        srv.close()
    lat2, wall2 = cox.percall_run_trace(items)
    assert min(lat2) > 0 and wall2 >= max(arrivals)


def test_bad_requests_are_rejected(cox):
    import torch
    srv = cox.Server(1 << 20)
    try:
        x = torch.zeros(16, dtype=torch.float32, device="cuda")
        r = cox.make_request(cox.COX_REQ_SCAN, x, width=3)
        with pytest.raises(cox.CoxError):
            srv.submit(r)
        r = cox.make_request(cox.COX_REQ_REDUCE, x.view(torch.int32), compensated=True)
        with pytest.raises(cox.CoxError):
            srv.submit(r)
        good = cox.make_request(cox.COX_REQ_REDUCE, x)
        with pytest.raises(cox.CoxError):  # one bad request: none of the group is queued
            srv.submit_many([good, r, good])
        assert srv.stats()["submitted"] == 0
    finally:
        srv.close()
