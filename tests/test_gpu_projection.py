"""The projection's screen division against IEEE division, on the GPU.

Every geometry kernel divides both clip coordinates of a point by w through
one reciprocal, y = RN(1/w) (one Newton step on the hardware estimate), and
corrects each quotient after Markstein (1990), for w in [2^-40, 2^40).  The
render parity tests show whole frames equal to the oracle's; these tests pin
the arithmetic itself through pcr_check_division:

- the reciprocal equals the IEEE one for every float in the window;
- the quotient equals IEEE c / w on dense grids of significands and on
  random bit patterns (all exponents, zeros, subnormals, infinities, NaNs);
- the screen coordinate equals the one from the IEEE quotient, or both are
  culled, for every pair.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_2104_07526_gb300 import pcr

pytestmark = pytest.mark.gpu

WINDOW_LO = 0x2B800000  # bits of 2^-40
WINDOW_HI = 0x53800000  # bits of 2^40
ONE = 0x3F800000


@pytest.fixture(scope="module")
def ctx():
    from gpu_helpers import ensure_built
    ensure_built()
    c = pcr.Context(0, stream=torch.cuda.current_stream())
    yield c.handle
    c.close()


def test_reciprocal_exact_over_the_whole_window(ctx):
    got = pcr.pcr_check_division(ctx, WINDOW_LO, WINDOW_HI - WINDOW_LO)
    assert got["reciprocal_mismatches"] == 0
    # the bit patterns just outside the window are skipped, not checked
    edge = pcr.pcr_check_division(ctx, WINDOW_LO - 1000, 2000)
    assert edge["reciprocal_mismatches"] == 0


def test_quotient_on_a_grid_of_significands(ctx):
    """w: 8 runs of 2^15 consecutive significands spread over [1, 2); c: every
    8th significand in [1, 2).  2^38 pairs; quotients in (0.5, 2) span both
    binades next to 1."""
    for k in range(8):
        got = pcr.pcr_check_division(ctx, ONE + k * (1 << 20), 1 << 15, c_first=ONE, c_count=1 << 20, c_step=8,
                                     size=1920.0)
        assert got["pairs"] == (1 << 15) * (1 << 20)
        assert got["quotient_pairs"] == got["pairs"]
        assert got["quotient_mismatches"] == 0
        assert got["screen_mismatches"] == 0


def test_quotient_on_random_and_special_numerators(ctx):
    rng = np.random.default_rng(20260301)
    c = rng.integers(0, 2**32, size=1 << 20, dtype=np.uint64).astype(np.uint32)
    special = np.array([0x00000000, 0x80000000, 0x00000001, 0x80000001, 0x007FFFFF, 0x00800000, 0x7F7FFFFF,
                        0xFF7FFFFF, 0x7F800000, 0xFF800000, 0x7FC00000, 0xFFC00000, 0x3F800000, 0xBF800000,
                        0x4F000000, 0x30800000, 0x2F800000, 0x2E800000], dtype=np.uint32)
    c[:special.size] = special
    dev = torch.from_numpy(c.view(np.int32)).cuda()
    total = {"quotient_mismatches": 0, "screen_mismatches": 0, "quotient_pairs": 0, "pairs": 0}
    starts = rng.integers(WINDOW_LO, WINDOW_HI - 64, size=24)
    for w0 in list(starts) + [WINDOW_LO, WINDOW_HI - 64, ONE - 32]:
        for size in (1920.0, 1080.0, 7.0):
            got = pcr.pcr_check_division(ctx, int(w0), 64, c_bits=dev, size=size)
            for k in total:
                total[k] += got[k]
    assert total["pairs"] == 27 * 3 * 64 * c.size
    assert total["quotient_pairs"] > total["pairs"] // 4
    assert total["quotient_mismatches"] == 0
    assert total["screen_mismatches"] == 0


def test_check_rejects_bad_arguments(ctx):
    with pytest.raises(pcr.PcrError):
        pcr.pcr_check_division(ctx, ONE, 1, c_first=ONE, c_count=4, c_step=0)
    with pytest.raises(pcr.PcrError):
        pcr.pcr_check_division(ctx, ONE, 1, size=0.0)
