"""FP64-definition checks for fp32 sums and scans computed on the GPU.

Every fp32 result is compared with the plain definition (the oracle's FP64
value r of the same inputs, and sum |x| over the inputs that feed it):

* compensated results: err = |y - r| / max(|r|, 2^-24 sum|x|) <= 1e-5 at
  every output (the stated tolerance; Ogita, Rump and Oishi bound the error
  of a compensated cascade by u|r| + gamma_h^2 sum|x|);
* plain results: |y - r| <= gamma_h * sum|x| with gamma_h = h u / (1 - h u),
  u = 2^-24, the textbook bound for any summation whose additions form a tree
  of depth h (Higham, "Accuracy and Stability of Numerical Algorithms",
  section 4.2).  h is the depth of the order the kernel states, so a dropped
  or doubled term, a wrong sign or a shifted segment fails it.

The helpers also return the error statistics, so a test can report them.
"""
from __future__ import annotations

import math

import numpy as np

TOL = 1e-5
U32 = 2.0 ** -24


def gamma(h: int) -> float:
    return h * U32 / (1.0 - h * U32)


def tile_depth(width: int) -> int:
    """Additions on the longest path of a width-`width` tree or Hillis-Steele scan."""
    return max(1, int(math.log2(width)))


def block_depth(width: int, block_dim: int) -> int:
    """Longest path of the stated BLOCK order: a width tree per tile, warp 0's
    lane l folding tile partials l, l+32, ... in turn, then a 32-wide tree."""
    partials = max(1, block_dim // width)
    return tile_depth(width) + max(0, -(-partials // 32) - 1) + 5


def stats(y, ref, ab) -> dict:
    """Error statistics of y against the FP64 definition: the tolerance metric
    (max), pointwise |y - r| / |r| over r != 0 (max, p99) and the normwise
    ||y - r||_2 / ||r||_2."""
    y = np.asarray(y, dtype=np.float64)
    d = np.abs(y - ref)
    den = np.maximum(np.abs(ref), U32 * ab)
    den = np.where(den == 0, 1.0, den)
    nz = ref != 0
    pw = d[nz] / np.abs(ref[nz]) if nz.any() else np.zeros(1)
    nr = float(np.linalg.norm(ref))
    return {"max_err": float((d / den).max()) if d.size else 0.0,
            "max_pointwise": float(pw.max()) if pw.size else 0.0,
            "p99_pointwise": float(np.percentile(pw, 99)) if pw.size else 0.0,
            "normwise": float(np.linalg.norm(y - ref) / nr) if nr > 0 else float(np.linalg.norm(y - ref))}


def assert_fp64(y, ref, ab, compensated: bool, depth: int, what: str = "") -> dict:
    """Asserts the FP64-definition bound for compensated or plain fp32 results."""
    y64 = np.asarray(y, dtype=np.float64)
    assert y64.shape == np.shape(ref), what
    s = stats(y64, ref, ab)
    if compensated:
        assert s["max_err"] <= TOL, f"{what}: compensated error {s['max_err']:.3e} > {TOL}"
    else:
        bound = gamma(depth) * np.asarray(ab, dtype=np.float64)
        bad = np.abs(y64 - ref) > bound
        assert not bad.any(), (f"{what}: plain result outside gamma_{depth} sum|x| at "
                               f"{int(np.flatnonzero(bad)[0])}")
    return s
