"""CPU-side checks of the C ABI: the library loads, exports every symbol the
headers declare, and rejects bad arguments on the host before any CUDA call.
No test here launches work (this file runs without a GPU)."""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cox():
    from paper_2112_10034_gb300 import build, cox as c
    build.build()
    return c


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(cox_[a-z0-9_]+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported(cox):
    lib = cox.lib()
    declared = _declared()
    assert len(declared) >= 10
    so = os.path.join(ROOT, "paper_2112_10034_gb300", "libcox.so")
    nm = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (cox_[a-z0-9_]+)", nm))
    assert declared <= exported, declared - exported
    for name in declared:
        assert hasattr(lib, name)


def test_binding_covers_the_header(cox):
    assert _declared() == set(cox.SIGNATURES)


def test_status_strings_and_version(cox):
    assert cox.cox_version() >= 100
    assert cox.status_string(cox.COX_OK) == "COX_OK"
    assert "timeout" in cox.status_string(cox.COX_ETIMEOUT).lower() or "wait" in cox.status_string(5)


def test_workspace_sizes(cox):
    assert cox.cox_tile_reduce_workspace(cox.COX_SCOPE_TILE, 10**6, 256) == 0
    assert cox.cox_tile_reduce_workspace(cox.COX_SCOPE_GRID, 10**6, 256) > 0
    tile = 8192
    # header + a descriptor per tile + a descriptor and an accumulator per group of 32 tiles
    t = 2**28 // tile
    assert cox.cox_ballot_compact_workspace(2**28, 256) == 256 + 8 * t + 16 * ((t + 31) // 32)
    assert cox.cox_ballot_compact_workspace(2**28, 1024) == 256 + 8 * t + 16 * ((t + 31) // 32)
    assert cox.cox_ballot_compact_workspace(1, 256) == 256 + 8 + 16


@pytest.mark.parametrize("width", [0, 1, 3, 64])
def test_bad_width_is_einval(cox, width):
    assert cox.cox_tile_scan(cox.COX_SUM, cox.COX_F32, width, 256, 16, 16, 10, 0, None) == cox.COX_EINVAL
    assert cox.cox_shfl(0, 0, width, 256, 16, 16, 10, 0, cox.FULL_MASK, None) == cox.COX_EINVAL


@pytest.mark.parametrize("block", [0, 31, 48, 1056])
def test_bad_block_is_einval(cox, block):
    assert cox.cox_tile_reduce(0, 0, 32, block, 1, 16, 16, 10, 0, None, None, 0, None) == cox.COX_EINVAL


def test_host_validation(cox):
    E = cox.COX_EINVAL
    # partial masks are outside the paper's non-divergent scope
    assert cox.cox_shfl(0, 0, 32, 256, 16, 16, 10, 0, 0x0000FFFF, None) == cox.COX_EUNSUPPORTED
    # delta out of range, bad function / dtype / op
    assert cox.cox_shfl(cox.COX_SHFL_UP, 0, 32, 256, 16, 16, 10, 32, cox.FULL_MASK, None) == E
    assert cox.cox_shfl(8, 0, 32, 256, 16, 16, 10, 0, cox.FULL_MASK, None) == E
    assert cox.cox_shfl(0, 3, 32, 256, 16, 16, 10, 0, cox.FULL_MASK, None) == E
    assert cox.cox_tile_scan(cox.COX_AND, cox.COX_F32, 32, 256, 16, 16, 10, 0, None) == E
    # compensation only for fp32 sums; fp64 combine only for compensated GRID
    assert cox.cox_tile_scan(cox.COX_SUM, cox.COX_I32, 32, 256, 16, 16, 10, cox.COX_F_COMPENSATED, None) == E
    assert cox.cox_tile_reduce(0, 2, 32, 256, 1, 16, 16, 10, cox.COX_F_FP64_COMBINE, None, None, 0, None) == E
    # null pointers and negative sizes
    assert cox.cox_tile_scan(0, 0, 32, 256, None, 16, 10, 0, None) == E
    assert cox.cox_tile_scan(0, 0, 32, 256, 16, 16, -1, 0, None) == E
    # compaction: float keys, missing count, too-small workspace
    assert cox.cox_ballot_compact(cox.COX_F32, 32, 256, 16, 10, 5, 16, 16, 16, 4096, 0, None) == E
    assert cox.cox_ballot_compact(0, 32, 256, 16, 10, 5, 16, None, 16, 4096, 0, None) == E
    assert cox.cox_ballot_compact(0, 32, 256, 16, 10, 5, 16, 16, 16, 8, 0, None) == cox.COX_ENOMEM
    # histogram bins range
    assert cox.cox_match_histogram(0, 32, 256, 16, 10, 0, 16, None, 0, None) == E
    assert cox.cox_match_histogram(0, 32, 256, 16, 10, 8193, 16, None, 0, None) == E
    assert cox.cox_match_histogram(0, 32, 256, 16, 10, 256, 16, None, 64, None) == E
    assert cox.cox_match_histogram(0, 32, 256, 16, 10, 256, 16, None, 8 | 32, None) == E
    assert cox.cox_match_histogram(0, 32, 256, 16, 10, 256, 16, None, 8 | 16, None) == E
