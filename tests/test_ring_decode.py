"""Host check of the halo-ring index decode of the blocked kernels (FP32 k_tb2d32 and FP64
k_tb2d use the same decode).

At step s of a launch of T steps the kernel updates the ring of radius
r = T - 1 - s around its BX x BY tile, enumerated by a flat index e; row and
column come from an integer division by the row length done as a 32-bit
multiply-high by ceil(2^32 / d).  This test replays that decode for every tile
shape and depth the library builds and checks that the ring is covered exactly
once and stays inside the extended tile (so every shared-memory access of the
kernel is in bounds), and checks the division itself exhaustively.  The FP64 kernels'
ring_coords and multiplier table are also cut out of the kernel source, compiled for the
host and held to the same coverage."""

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


# ---- the kernel source itself, compiled for the host --------------------------------------

def _extract(text, start, end_marker=None):
    """The source from `start` to the end of its brace block (or to end_marker)."""
    i = text.index(start)
    if end_marker is not None:
        return text[i:text.index(end_marker, i) + len(end_marker)]
    depth, j = 0, text.index("{", i)
    for k in range(j, len(text)):
        depth += {"{": 1, "}": -1}.get(text[k], 0)
        if depth == 0:
            return text[i:k + 1]
    raise ValueError(start)


def test_kernel_ring_coords_cover_each_point_once(tmp_path):
    """ring_coords and the multiplier table of the FP64 blocked kernels (wave_tb_kernels.cuh),
    cut out of the kernel source and compiled for the host (__umulhi written out as the high
    word of the 64-bit product), cover every ring point of every radius exactly once and stay
    inside the extended tile, for every depth and tile height of the blocked kernels."""
    import ctypes
    import os
    import shutil
    import subprocess
    if shutil.which("g++") is None:
        pytest.skip("no host C++ compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with open(os.path.join(root, "paper_2507_23613_gb300", "csrc", "wave_tb_kernels.cuh")) as fh:
        text = fh.read()
    table = _extract(text, "struct DivMagic {",
                     "__device__ __forceinline__ unsigned div_magic(int d) { return c_div_magic.m[d]; }")
    coords = _extract(text, "template <int T, int BX, int BY>\n__device__ __forceinline__ void ring_coords(")
    cases = [(T, by) for T in (2, 3, 4, 8) for by in sorted(set(SHAPES))]
    body = "\n".join(
        f"  if (T == {T} && BY == {by}) return check<{T}, {by}>();" for T, by in cases)
    src = f"""
#include <cstdint>
#include <vector>
#define __device__
#define __forceinline__ inline
#define __constant__ static
static inline unsigned __umulhi(unsigned a, unsigned b) {{
  return (unsigned)(((unsigned long long)a * b) >> 32);
}}
{table}
{coords}
template <int T, int BY>
long check() {{
  constexpr int BX = {BX}, EX = BX + 2 * T, EY = BY + 2 * T;
  long bad = 0;
  for (int r = 1; r < T; ++r) {{
    const int rw = BX + 2 * r, top = 2 * r * rw, ring = top + 2 * r * BY;
    std::vector<int> hits(EX * EY, 0);
    for (int e = 0; e < ring; ++e) {{
      int lx, ly;
      ring_coords<T, BX, BY>(e, r, rw, top, div_magic(rw), div_magic(2 * r), lx, ly);
      if (lx < 1 || lx > EX - 2 || ly < 1 || ly > EY - 2) {{ ++bad; continue; }}
      ++hits[ly * EX + lx];
    }}
    for (int y = 0; y < EY; ++y)
      for (int x = 0; x < EX; ++x) {{
        const bool in_box = x >= T - r && x < T + BX + r && y >= T - r && y < T + BY + r;
        const bool in_tile = x >= T && x < T + BX && y >= T && y < T + BY;
        bad += hits[y * EX + x] != ((in_box && !in_tile) ? 1 : 0);
      }}
  }}
  return bad;
}}
extern "C" long ring_violations(int T, int BY) {{
{body}
  return -1;
}}
"""
    cpp, so = tmp_path / "ring.cpp", tmp_path / "libring.so"
    cpp.write_text(src)
    subprocess.run(["g++", "-std=c++17", "-O1", "-shared", "-fPIC", str(cpp), "-o", str(so)],
                   check=True, capture_output=True)
    lib = ctypes.CDLL(str(so))
    lib.ring_violations.restype = ctypes.c_long
    lib.ring_violations.argtypes = [ctypes.c_int, ctypes.c_int]
    for T, by in cases:
        assert lib.ring_violations(T, by) == 0, (T, by)
