"""The Rys quadrature tables used by the library's Rys kernels (written by
csrc/gen_rys.py), evaluated here the way the device evaluates them, against
the definition of the rule: for the n-point rule at T,
    sum_i w_i u_i^k = F_k(T)  for k = 0 .. 2n-1
(F_k the Boys function, here the oracle's, itself pinned to the incomplete
gamma function), on T inside every table interval and past the switch to the
large-T limit."""
import os
import re

import numpy as np
import pytest

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1708_00033_gb300", "csrc",
                   "rys_tables.h")


def _tables():
    txt = open(HDR).read()
    deg = int(re.search(r"kRysDeg = (\d+);", txt).group(1))
    nmax = int(re.search(r"kRysMaxRoots = (\d+);", txt).group(1))
    sw = dict((int(a), int(b)) for a, b in re.findall(r"n == (\d+) \? (\d+)", txt))
    out = {}
    for n in range(1, nmax + 1):
        def arr(name):
            body = re.search(name + r"\[\d+\] = \{(.*?)\};", txt, re.S).group(1)
            return np.array([float(x) for x in body.replace("\n", " ").split(",") if x.strip()])
        out[n] = (arr(f"kRysTab{n}"), arr(f"kRysHermX{n}"), arr(f"kRysHermW{n}"), sw[n])
    return deg, out


def _rule(deg, tab, hx, hw, sw, n, T):
    """Nodes and weights as rys_rule<n> computes them (Horner in x = 2 (T - k) - 1)."""
    if T < sw:
        k = int(T)
        x = 2.0 * (T - k) - 1.0
        c = tab[k * 2 * n * (deg + 1):(k + 1) * 2 * n * (deg + 1)].reshape(2 * n, deg + 1)
        v = np.zeros(2 * n)
        for i in range(2 * n):
            acc = c[i, deg]
            for j in range(deg - 1, -1, -1):
                acc = acc * x + c[i, j]
            v[i] = acc
        return v[:n], v[n:]
    rs = 1.0 / np.sqrt(T)
    return hx * rs * rs, hw * rs


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_rys_rule_reproduces_boys_moments(oracle_mod, n):
    deg, tabs = _tables()
    tab, hx, hw, sw = tabs[n]
    rng = np.random.default_rng(n)
    Ts = list(np.concatenate([rng.uniform(0, sw, 40), [0.0, 1e-9, sw - 1e-9, float(sw), sw + 0.5, 80.0, 400.0]]))
    worst = 0.0
    for T in Ts:
        u, w = _rule(deg, tab, hx, hw, sw, n, T)
        assert np.all(u > 0) and np.all(u < 1) and np.all(np.diff(u) > 0) and np.all(w > 0)
        F = oracle_mod.boys(2 * n - 1, T)
        for k in range(2 * n):
            rel = abs(np.sum(w * u ** k) / F[k] - 1.0)
            worst = max(worst, rel)
    assert worst <= 2e-14, worst
