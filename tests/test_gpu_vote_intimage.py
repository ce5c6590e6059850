"""GPU parity of the second-workload row: batched vote statistics (the SDK's
VoteAny/VoteAll kernels as per-segment any/all/popcount counts over tile
ballots) and batched integral images (row shuffle scans plus column sums).
Both are integer results and must equal the oracle exactly."""
import numpy as np
import pytest

import oracle as o
from paper_2112_10034_gb300 import inputs

pytestmark = pytest.mark.gpu
WIDTHS = [2, 4, 8, 16, 32]


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


@pytest.mark.parametrize("W", WIDTHS)
@pytest.mark.parametrize("density", [0.0, 0.05, 0.5, 0.97, 1.0])
def test_vote_stats(cox, W, density):
    import torch
    for n, seg in ((1, 32), (1000, 64), (70_001, 1024), (70_001, 4096 + 32), (1 << 20, 16384), (5000, W),
                   (70_001, 4096), ((1 << 20) + 77, 8192)):  # 16384, 4096, 8192: the 128-bit-load kernel
        thr = inputs.density_threshold(density) if density < 1 else 2**31
        pred = (inputs.uniform_u31(n, seed=n + W) < thr).astype(np.int32) * \
            (1 + (inputs.bits_u32(n, seed=n) & 7).astype(np.int32))
        nseg = (n + seg - 1) // seg
        st = torch.full((nseg * 3 + 4,), -1, dtype=torch.int64, device="cuda")
        assert cox.cox_vote_stats(o.I32, W, dev(pred).data_ptr(), n, seg, st.data_ptr(), None) == 0
        got = st.cpu().numpy()
        np.testing.assert_array_equal(got[:nseg * 3].reshape(nseg, 3), o.vote_stats(W, pred, seg),
                                      err_msg=f"n={n} seg={seg}")
        assert (got[nseg * 3:] == -1).all()


def test_vote_stats_fp32_zeros_and_bad_args(cox):
    import torch
    f = inputs.normal_f32(4096, seed=2)
    f[::3] = 0.0
    f[1::5] = -0.0
    st = torch.zeros(3 * 4, dtype=torch.int64, device="cuda")
    assert cox.cox_vote_stats(o.F32, 8, dev(f).data_ptr(), 4096, 1024, st.data_ptr(), None) == 0
    want = o.vote_stats(8, (f != 0).astype(np.int32), 1024)
    np.testing.assert_array_equal(st.cpu().numpy().reshape(4, 3), want)
    assert cox.cox_vote_stats(o.I32, 8, dev(f).data_ptr(), 4096, 1020, st.data_ptr(), None) == cox.COX_EINVAL
    assert cox.cox_vote_stats(o.I32, 3, dev(f).data_ptr(), 4096, 1024, st.data_ptr(), None) == cox.COX_EINVAL


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 7, 5), (3, 33, 31), (2, 64, 64), (4, 100, 1000),
                                   (2, 1080, 1920), (1, 17, 4097), (3, 130, 1040), (1, 700, 2048),
                                   (2, 65, 16), (2, 3, 132), (1, 64, 528), (5, 129, 4),
                                   # enough 128-column strips for the strip walk: ragged strips and
                                   # stages, several units per warp, more than 32 strips per row
                                   (64, 70, 1920), (640, 37, 272), (40, 100, 3840), (40, 20, 4224)])
@pytest.mark.parametrize("dt", ["u8", "u32"])
def test_integral_image(cox, shape, dt):
    import torch
    b, h, w = shape
    bits = inputs.bits_u32(b * h * w, seed=b * h * w + len(dt))
    img = (bits & 0xFF).astype(np.uint8).reshape(shape) if dt == "u8" else bits.reshape(shape)
    code = cox.COX_U8 if dt == "u8" else cox.COX_U32
    out = torch.full((b * h * w + 16,), 0x7FBADBAD, dtype=torch.int32, device="cuda")
    wsb = cox.cox_integral_image_workspace(b, h, w)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    d_in = dev(img.view(np.uint8).ravel() if dt == "u8" else img.view(np.int32).ravel())
    assert cox.cox_integral_image(code, b, h, w, d_in.data_ptr(), out.data_ptr(), ws.data_ptr(), wsb, None) == 0
    got = out.cpu().numpy()
    np.testing.assert_array_equal(got[:b * h * w].view(np.uint32).reshape(shape), o.integral_image(img))
    assert (got[b * h * w:] == 0x7FBADBAD).all()


@pytest.mark.parametrize("dt", ["u8", "u32"])
@pytest.mark.parametrize("in_off,out_off", [(1, 0), (0, 1), (4, 2)])
def test_integral_image_misaligned(cox, dt, in_off, out_off):
    """Input or output off the 16-byte grid takes the three-pass form."""
    import torch
    b, h, w = 2, 70, 1040
    bits = inputs.bits_u32(b * h * w, seed=77 + in_off)
    img = (bits & 0xFF).astype(np.uint8).reshape(b, h, w) if dt == "u8" else bits.reshape(b, h, w)
    code = cox.COX_U8 if dt == "u8" else cox.COX_U32
    esz = 1 if dt == "u8" else 4
    raw = img.view(np.uint8).ravel()
    d_in = torch.zeros(raw.size + 64, dtype=torch.uint8, device="cuda")
    d_in[in_off * esz:in_off * esz + raw.size] = torch.from_numpy(raw).cuda()
    out = torch.full((b * h * w + 16,), 0x7FBADBAD, dtype=torch.int32, device="cuda")
    wsb = cox.cox_integral_image_workspace(b, h, w)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    assert cox.cox_integral_image(code, b, h, w, d_in.data_ptr() + in_off * esz, out.data_ptr() + 4 * out_off,
                                  ws.data_ptr(), wsb, None) == 0
    got = out.cpu().numpy()
    np.testing.assert_array_equal(got[out_off:out_off + b * h * w].view(np.uint32).reshape(b, h, w),
                                  o.integral_image(img))
    assert (got[:out_off] == 0x7FBADBAD).all() and (got[out_off + b * h * w:] == 0x7FBADBAD).all()


@pytest.mark.parametrize("dt", ["u8", "u32"])
def test_integral_image_strip_walk_reuses_its_workspace(cox, dt):
    """Two calls in a row on one workspace (the strip counters restart at 0
    each call), the second on other pixels."""
    import torch
    b, h, w = 96, 45, 1040
    code = cox.COX_U8 if dt == "u8" else cox.COX_U32
    wsb = cox.cox_integral_image_workspace(b, h, w)
    ws = torch.full((wsb,), 0xFF, dtype=torch.uint8, device="cuda")
    for seed in (5, 6):
        bits = inputs.bits_u32(b * h * w, seed=seed)
        img = (bits & 0xFF).astype(np.uint8).reshape(b, h, w) if dt == "u8" else bits.reshape(b, h, w)
        d_in = dev(img.view(np.uint8).ravel() if dt == "u8" else img.view(np.int32).ravel())
        out = torch.empty(b * h * w, dtype=torch.int32, device="cuda")
        assert cox.cox_integral_image(code, b, h, w, d_in.data_ptr(), out.data_ptr(), ws.data_ptr(), wsb, None) == 0
        np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32).reshape(b, h, w), o.integral_image(img))
    assert cox.cox_device_status(None) == cox.COX_OK
