"""The batched kernels map a block to its tile with t / d and t % d computed
from the FP32 reciprocal of d and one correction (tile_divmod in
csrc/lb_batch.cuh).  The same FP32 arithmetic, emulated here with numpy, is
exact for every block index t < 2^24 (the largest lattice has < 2^23 tiles
or warp segments) and a spread of divisors."""
import numpy as np
import pytest


@pytest.mark.parametrize("d", [1, 2, 3, 7, 8, 31, 33, 127, 128, 1000, 4097, 65535, 131071,
                               524287, 8388607, 16777215])
def test_reciprocal_divmod_is_exact_below_2_24(d):
    t = np.arange(1 << 24, dtype=np.int64)
    inv = np.float32(1.0) / np.float32(d)
    q = np.trunc(t.astype(np.float32) * inv).astype(np.int64)   # fl32 product, then truncation
    r = t - q * d
    q = np.where(r < 0, q - 1, np.where(r >= d, q + 1, q))
    assert np.array_equal(q, t // d)
