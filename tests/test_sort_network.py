"""The integer logic of the warp-local quartet sort of the FP64 ERI launches, emulated on the CPU.

Each warp writes one key per quartet of its window (staircase length << 16 | position), sorts the window
with a bitonic network whose compare-exchange pairs are lo = 2i - (i & (stride - 1)), hi = lo + stride for
i < n/2 (ascending where lo & size == 0), and runs the sorted positions in rounds.  This checks that the
network sorts every window size the kernels use and that every position is visited exactly once, and that
the window-size rule gives each warp at least two windows.  The device code itself runs in every GPU test."""
import numpy as np
import pytest

SORT_ROUNDS = 8


def _bitonic(keys):
    k = list(keys)
    n = len(k)
    size = 2
    while size <= n:
        stride = size >> 1
        while stride > 0:
            for i in range(n >> 1):
                lo = 2 * i - (i & (stride - 1))
                hi = lo + stride
                assert 0 <= lo < hi < n
                x, y = k[lo], k[hi]
                if (x > y) == ((lo & size) == 0):
                    k[lo], k[hi] = y, x
            stride >>= 1
        size <<= 1
    return k


@pytest.mark.parametrize("n", [2, 4, 8, 16, 32, 64, 128, 256])
def test_bitonic_network_sorts_every_window(n):
    rng = np.random.default_rng(n)
    for trial in range(20):
        lengths = rng.integers(0, 82 if trial % 2 else 4, n)  # staircases of 0..81, or many ties
        keys = [(int(t) << 16) | pos for pos, t in enumerate(lengths)]
        out = _bitonic(keys)
        assert out == sorted(keys)
        assert sorted(x & 0xFFFF for x in out) == list(range(n))


def _rounds(n_quartets, nwarps, gpw):
    R = 1
    while R < SORT_ROUNDS and 2 * R * gpw * nwarps * 2 <= n_quartets:
        R *= 2
    return R


@pytest.mark.parametrize("gk", [1, 2, 4, 8])
def test_window_rule(gk):
    gpw = 32 // gk
    nwarps = 152 * 16 * 4
    for n in [0, 1, 1000, gpw * nwarps * 4 - 1, gpw * nwarps * 4, 10 ** 6, 10 ** 8]:
        R = _rounds(n, nwarps, gpw)
        W = R * gpw
        assert R in (1, 2, 4, 8) and W <= SORT_ROUNDS * gpw
        assert W <= 0xFFFF
        if R > 1:
            assert n >= 2 * W * nwarps  # every warp gets at least two windows
