"""Host check of the halo-ring index decode of the blocked kernels (FP32 k_tb2d32 and FP64
k_tb2d use the same decode).

At step s of a launch of T steps the kernel updates the ring of radius
r = T - 1 - s around its BX x BY tile, enumerated by a flat index e; row and
column come from an integer division by the row length done as a 32-bit
multiply-high by ceil(2^32 / d).  This test replays that decode for every tile
shape and depth the library builds and checks that the ring is covered exactly
once and stays inside the extended tile (so every shared-memory access of the
kernel is in bounds), and checks the division itself exhaustively."""

import numpy as np
import pytest

BX = 32
SHAPES = [16 * 2, 16 * 1, 32 * 1, 16 * 4, 16 * 2]   # BY of the FP32 tile shapes 0-2 (K = 2 or 1)
SHAPES += [16 * 4, 16 * 2, 16 * 3, 8 * 4, 16 * 1]   # BY of the FP64 tile shapes 0-4


def div_magic(d):
    """The kernels' multiplier: 0xFFFFFFFF / d + 1 in unsigned 32-bit arithmetic."""
    return (0xFFFFFFFF // d + 1) & 0xFFFFFFFF


def umulhi(a, b):
    return (a * b) >> 32


def decode(e, r, T, BY):
    RW = BX + 2 * r
    top = 2 * r * RW
    if e < top:
        row = umulhi(e, div_magic(RW))
        lx = T - r + (e - row * RW)
        ly = T - r + row if row < r else T + BY + row - r
    else:
        e2 = e - top
        row = umulhi(e2, div_magic(2 * r))
        col = e2 - row * 2 * r
        ly = T + row
        lx = T - r + col if col < r else T + BX + col - r
    return lx, ly


@pytest.mark.parametrize("T", [2, 3, 4, 8, 16])
@pytest.mark.parametrize("BY", sorted(set(SHAPES)))
def test_ring_decode_covers_each_point_once(T, BY):
    EX, EY = BX + 2 * T, BY + 2 * T
    for r in range(1, T):
        ring = 2 * r * (BX + 2 * r) + 2 * r * BY
        seen = set()
        for e in range(ring):
            lx, ly = decode(e, r, T, BY)
            assert 1 <= lx <= EX - 2 and 1 <= ly <= EY - 2
            seen.add((lx, ly))
        want = {(x, y) for x in range(T - r, T + BX + r) for y in range(T - r, T + BY + r)
                if not (T <= x < T + BX and T <= y < T + BY)}
        assert len(seen) == ring and seen == want


def test_division_by_multiplier_is_exact():
    """floor(e / d) == (e * ceil(2^32 / d)) >> 32 for every ring index and divisor in use
    (indices below 2^16, divisors 2 .. 127), including powers of two."""
    e = np.arange(1 << 16, dtype=np.uint64)
    for d in range(2, 128):
        m = np.uint64(div_magic(d))
        assert np.array_equal((e * m) >> np.uint64(32), e // np.uint64(d)), d
