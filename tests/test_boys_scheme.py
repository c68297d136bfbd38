"""The FP64 Boys evaluation scheme of the ERI kernels, emulated on the CPU with exact table values, against
the oracle's Boys function (itself pinned to the incomplete gamma function).

The device builds its table at run time, so this test checks the scheme rather than the table bytes: the
row grids, the five-term Taylor chains, the region boundary at T = 64 and the row of T >= 64 taken from
T's bit pattern rounded to 12 mantissa bits, the asymptotic form's coefficients in that region, and the
downward recursion for L >= 2.  The table values at the grid points come from the oracle (region A) and
from the asymptotic form F_m(T) = (2m-1)!! / 2^(m+1) sqrt(pi / T^(2m+1)) (region B).  The device code
itself is covered end to end by the GPU parity tests."""
import math
import struct

import numpy as np
import pytest

SUB_BITS = 12  # rows per binade in region B: 2^12


def _bits(x: float) -> int:
    return struct.unpack("<q", struct.pack("<d", x))[0]


def _double(b: int) -> float:
    return struct.unpack("<d", struct.pack("<q", b))[0]


def _row(oracle_mod, T: float):
    """(T_k, F_0..F_12 at T_k, e^{-T_k}) of the row the kernels use for T."""
    if _bits(T) >= _bits(64.0):
        rb = _bits(T) + (1 << (51 - SUB_BITS))
        Tk = _double(rb & ~((1 << (52 - SUB_BITS)) - 1))
        F = [0.5 * math.sqrt(math.pi / Tk)]
        for m in range(12):
            F.append(F[m] * (2 * m + 1) / (2.0 * Tk))
        return Tk, np.array(F), 0.0
    Tk = round(T * 512.0) / 512.0
    return Tk, np.asarray(oracle_mod.boys(12, Tk)), math.exp(-Tk)


def _eval(oracle_mod, L: int, T: float) -> np.ndarray:
    Tk, F, e = _row(oracle_mod, T)
    d = Tk - T
    fact = [1.0, 1.0, 2.0, 6.0, 24.0]

    def horner(c):
        return c[0] + d * (c[1] + d * (c[2] + d * (c[3] + d * c[4])))

    out = np.zeros(L + 1)
    if L <= 1:
        for m in range(L + 1):
            out[m] = horner([F[m + j] / fact[j] for j in range(5)])
    else:
        out[L] = horner([F[L + j] / fact[j] for j in range(5)])
        ex = horner([e / fact[j] for j in range(5)])
        for m in range(L - 1, -1, -1):
            out[m] = (2.0 * T * out[m + 1] + ex) / (2 * m + 1)
    return out


def test_region_b_rows_from_bits():
    """The row of T >= 64 is T rounded to 12 mantissa bits, so |T - T_k| <= T / 8192, and T_k is a grid point
    2^e (1 + i / 4096); rounding up across a binade boundary lands on the next binade's first row."""
    rng = np.random.default_rng(0)
    for T in list(rng.uniform(64, 2 ** 31, 2000)) + [64.0, 128.0 - 1e-9, 2.0 ** 31 - 1.0]:
        rb = _bits(T) + (1 << (51 - SUB_BITS))
        Tk = _double(rb & ~((1 << (52 - SUB_BITS)) - 1))
        assert abs(Tk - T) <= T / 8192 * (1 + 1e-12)
        e = math.floor(math.log2(Tk))
        i = (Tk / 2.0 ** e - 1.0) * 4096
        assert abs(i - round(i)) == 0 and 0 <= round(i) < 4096 and 6 <= e <= 31


@pytest.mark.parametrize("L", [0, 1, 2, 4, 8])
def test_fp64_boys_scheme_vs_oracle(oracle_mod, L):
    rng = np.random.default_rng(10 + L)
    Ts = np.concatenate([rng.uniform(0, 64, 120), 10 ** rng.uniform(math.log10(64), 9.3, 120),
                         [0.0, 1e-12, 1.0 / 1024, 36.0, 59.0, 63.999999, 64.0, 64.000001, 127.99999, 2.0 ** 31 - 10]])
    worst = 0.0
    for T in Ts:
        got = _eval(oracle_mod, L, float(T))
        ref = np.asarray(oracle_mod.boys(L, float(T)))
        worst = max(worst, float(np.max(np.abs(got - ref) / ref)))
    assert worst < 2e-15, worst
