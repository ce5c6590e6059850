"""CPU checks of the FP64-definition bounds used by the GPU tests.

The oracle's fp32 emulations of the stated association orders must sit
inside the tree-depth bound gamma_h sum|x| (plain) and the 1e-5 tolerance
(compensated) for every width and block size the GPU tests use, and a planted
mistake -- one input dropped, one segment shifted -- must fail the bound.
"""
import numpy as np
import pytest

import oracle as o
from paper_2112_10034_gb300 import inputs
from tests import fpcheck as fc


@pytest.mark.parametrize("W", [2, 4, 8, 16, 32])
@pytest.mark.parametrize("B", [32, 96, 256, 1024])
def test_emulated_orders_meet_the_bounds(W, B):
    n = B * 40 + 13
    x = inputs.normal_f32(n, seed=W * 7 + B)
    for scope, seg in ((o.TILE, W), (o.BLOCK, B)):
        _, ref, ab = o.reduce_ref(o.SUM, o.F32, seg, x)
        depth = fc.tile_depth(W) if scope == o.TILE else fc.block_depth(W, B)
        for comp in (False, True):
            y, _ = o.reduce_emulate(o.SUM, o.F32, W, B, scope, x, comp)
            fc.assert_fp64(y, ref, ab, comp, depth, f"scope={scope} comp={comp}")
    _, ref, ab = o.scan_ref(o.SUM, o.F32, W, x)
    for comp in (False, True):
        fc.assert_fp64(o.scan_emulate(o.SUM, o.F32, W, B, x, comp), ref, ab, comp, fc.tile_depth(W))


def test_planted_mistakes_fail_the_bounds():
    W, B = 32, 256
    x = inputs.normal_f32(B * 20, seed=5)
    _, ref, ab = o.reduce_ref(o.SUM, o.F32, B, x)
    y, _ = o.reduce_emulate(o.SUM, o.F32, W, B, o.BLOCK, x)
    bad = y.copy()
    bad[3] -= x[3 * B + 17]  # one input dropped from block 3
    with pytest.raises(AssertionError):
        fc.assert_fp64(bad, ref, ab, False, fc.block_depth(W, B))
    with pytest.raises(AssertionError):
        fc.assert_fp64(bad, ref, ab, True, fc.block_depth(W, B))
    _, sref, sab = o.scan_ref(o.SUM, o.F32, W, x)
    s = o.scan_emulate(o.SUM, o.F32, W, B, x)
    shifted = np.roll(s, 1)  # every output one position late
    with pytest.raises(AssertionError):
        fc.assert_fp64(shifted, sref, sab, False, fc.tile_depth(W))


def test_stats_closed_forms():
    ref = np.array([1.0, -2.0, 0.0, 4.0])
    ab = np.array([1.0, 2.0, 8.0, 4.0])
    y = np.array([1.0, -2.0, 2.0 ** -30, 4.0 * (1 + 2.0 ** -20)])
    s = fc.stats(y, ref, ab)
    assert s["max_pointwise"] == pytest.approx(2.0 ** -20)
    # the zero reference uses the floor u * sum|x| = 2^-21: 2^-30 / 2^-21
    assert s["max_err"] == pytest.approx(2.0 ** -9)
    assert s["normwise"] == pytest.approx(np.hypot(2.0 ** -30, 4.0 * 2.0 ** -20) / np.sqrt(21.0))
    assert fc.gamma(1) == pytest.approx(2.0 ** -24 / (1 - 2.0 ** -24))
