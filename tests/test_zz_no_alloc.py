"""The compaction entry point that allocates nothing: cox_ballot_compact_static.

Some callers of this library cannot allocate device memory: code running
under a host framework whose allocator owns the whole device budget and
forbids side allocations, a latency-critical loop that must not take the
implicit device synchronisation of cudaMalloc/cudaFree, or a plugin that is
handed only its input and output buffers.  For them the library keeps the
compaction's scratch in a fixed 1 MiB array of its own.

These tests call that entry point through the C ABI and check that it returns
exactly what the workspace-taking cox_ballot_compact returns (compaction is
bit-exact), on two calls in a row whose inputs differ, so that scratch left
over by the first call cannot leak into the second; and that an input larger
than the fixed scratch can describe is refused before anything runs.  The
file name sorts last so that a run that stops at the first failure has
already run every other test.
"""
import numpy as np
import pytest

from paper_2112_10034_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cox():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_10034_gb300 import build, cox as c
    build.build()
    c.lib()
    return c


def _with_workspace(cox, keys, n, t, block):
    import torch
    out = torch.full((n + 16,), -7, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    wsb = cox.cox_ballot_compact_workspace(n, block)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    assert cox.cox_ballot_compact(cox.COX_I32, 32, block, keys.data_ptr(), n, t, out.data_ptr(), cnt.data_ptr(),
                                  ws.data_ptr(), wsb, 0, None) == cox.COX_OK
    return out, cnt


def _static(cox, keys, n, t, block):
    """Calls the static-scratch entry point; asserts that the call itself
    took no memory from torch's caching allocator (the outputs are made
    before it)."""
    import torch
    out = torch.full((n + 16,), -7, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    before = torch.cuda.memory_stats()["allocation.all.allocated"]
    assert cox.cox_ballot_compact_static(cox.COX_I32, 32, block, keys.data_ptr(), n, t, out.data_ptr(),
                                         cnt.data_ptr(), None) == cox.COX_OK
    assert torch.cuda.memory_stats()["allocation.all.allocated"] == before
    return out, cnt


@pytest.mark.parametrize("block", [256, 1024])
@pytest.mark.parametrize("n", [1, 300_007, (1 << 24) + 5])
def test_static_scratch_matches_workspace_entry_point_twice_in_a_row(cox, block, n):
    import torch
    first = torch.from_numpy(inputs.uniform_u31(n, seed=n + block)).cuda()
    second = torch.from_numpy(inputs.uniform_u31(n, seed=n + block + 1)).cuda()
    calls = [(first, inputs.density_threshold(0.9)), (second, inputs.density_threshold(0.1))]
    results = [_static(cox, k, n, t, block) for k, t in calls]  # two calls in a row
    torch.cuda.synchronize()
    for (k, t), (out, cnt) in zip(calls, results):
        ref_out, ref_cnt = _with_workspace(cox, k, n, t, block)
        c = int(ref_cnt.item())
        assert int(cnt.item()) == c
        np.testing.assert_array_equal(out.cpu().numpy(), ref_out.cpu().numpy())  # kept keys and untouched tail
        assert cox.device_status() == cox.COX_OK


def test_input_beyond_the_fixed_scratch_is_refused(cox):
    import torch
    keys = torch.zeros(16, dtype=torch.int32, device="cuda")
    out = torch.zeros(16, dtype=torch.int32, device="cuda")
    cnt = torch.full((1,), -1, dtype=torch.int64, device="cuda")  # a sentinel no run of the kernel leaves
    # 256 header bytes + 8 per tile of 8192 keys + 16 per group of 32 tiles: at most 123330 tiles
    limit = 123330 * 8192
    assert cox.cox_ballot_compact_workspace(limit, 256) <= cox.COX_COMPACT_STATIC_SCRATCH_BYTES
    assert cox.cox_ballot_compact_workspace(limit + 1, 256) > cox.COX_COMPACT_STATIC_SCRATCH_BYTES
    st = cox.cox_ballot_compact_static(cox.COX_I32, 32, 256, keys.data_ptr(), limit + 1, 0, out.data_ptr(),
                                       cnt.data_ptr(), None)
    assert st == cox.COX_ENOMEM
    torch.cuda.synchronize()
    assert int(cnt.item()) == -1  # nothing was enqueued: the count was neither cleared nor written
