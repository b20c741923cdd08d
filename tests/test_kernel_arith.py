"""Integer arithmetic the kernels take from FP32, checked on the CPU.

The candidate enumeration and the evaluation find a line's (iy, iz) from its
index l as the quotient and remainder of l by the lines per plane, nyb.  For
l below the bound the kernel states, they take the FP32 product l * rn(1/nyb),
truncate it, and correct the result by one step in either direction from the
remainder.  This replays that arithmetic with numpy's IEEE FP32 (the same
rounding) against integer division, over every small case and a random
sample of large ones, including exact multiples of nyb and their neighbours."""
import os
import re

import numpy as np

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_0908_4417_gb300", "csrc")


def kernel_bound():
    src = open(os.path.join(CSRC, "dsc_kernels.cu")).read()
    m = re.search(r"if \(l < \(1 << (\d+)\)\) \{\s*q = \(int\)\(\(float\)l \* inv_nyb\);", src)
    assert m, "line_yz's FP32 quotient not found"
    return 1 << int(m.group(1))


def quotient(l, nyb):
    inv = np.float32(1.0) / np.float32(nyb)                     # __frcp_rn: correctly rounded
    q = (l.astype(np.float32) * inv).astype(np.float32).astype(np.int64)
    r = l - q * nyb
    q = np.where(r < 0, q - 1, np.where(r >= nyb, q + 1, q))
    return q


def test_fp32_quotient_with_one_correction_is_exact():
    bound = kernel_bound()
    assert bound <= 1 << 23
    rng = np.random.default_rng(20090908)
    nybs = np.concatenate([np.arange(1, 3000), rng.integers(3000, 1 << 20, 3000)])
    raw_off = 0
    for nyb in nybs:
        mult = np.arange(1, 1500, dtype=np.int64) * nyb
        l = np.concatenate([np.arange(0, 2048), rng.integers(0, bound, 2000), mult, mult - 1, mult + 1,
                            [bound - 1]]).astype(np.int64)
        l = l[(l >= 0) & (l < bound)]
        inv = np.float32(1.0) / np.float32(nyb)
        raw = (l.astype(np.float32) * inv).astype(np.float32).astype(np.int64)
        raw_off = max(raw_off, int(np.abs(raw - l // nyb).max()))
        assert np.array_equal(quotient(l, nyb), l // nyb), nyb
    assert raw_off <= 1
