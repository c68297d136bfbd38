"""Generator of the per-angular-class ERI + J/K digestion kernels.

For every shell-quartet class (ab|cd) with l_a >= l_b, l_c >= l_d, l <= 2 and
bra pair class >= ket pair class (21 classes) this emits straight-line CUDA:

  per primitive quartet
    Boys F_m(T), m <= L = l_a+l_b+l_c+l_d, from a Taylor table (eri_common.cuh);
    [00|00]^(m) = prefactor * F_m(T);
    Obara-Saika vertical recurrence on electron 1
      [e+1_i 0|00]^(m) = PA_i [e0|00]^(m) + WP_i [e0|00]^(m+1)
                         + e_i/(2p) ([e-1_i 0|00]^(m) - rho/p [e-1_i 0|00]^(m+1))
    and on electron 2
      [e0|f+1_i 0]^(m) = QC_i [e0|f0]^(m) + WQ_i [e0|f0]^(m+1)
                         + f_i/(2q) ([e0|f-1_i 0]^(m) - rho/q [e0|f-1_i 0]^(m+1))
                         + e_i/(2(p+q)) [e-1_i 0|f0]^(m+1)
    up to the targets [e0|f0]^(0), l_a <= |e| <= l_a+l_b, l_c <= |f| <= l_c+l_d,
    accumulated over primitives (contraction before the horizontal step);
  per contracted quartet
    Head-Gordon-Pople horizontal recurrence (a b+1_i| = (a+1_i b| + AB_i (a b|,
    and the same on the ket with CD = C - D;
    digestion of the block X into the six Fock updates of Eq. 1a-1f with the
    unique-quartet weight f:  Jt_AB += 4f X.P_CD, Jt_CD += 4f X.P_AB,
    Kt_AC += 2f X.P_BD, Kt_BD += 2f X.P_AC, Kt_AD += 2f X.P_BC, Kt_BC += 2f X.P_AD,
    flushed with FP64 atomics (red.global.add.f64).

Only intermediates reachable from the targets are emitted, so each class does
the minimum recurrence work for its angular momenta.  The generator also
counts the floating-point operations per primitive quartet and per
contracted quartet; the library reports algorithmic FLOPs from these counts.

The emitted code is a template on the arithmetic type; it is instantiated for
double (the FP64 path) and float (small quartets of the mixed path, which
still accumulate into FP64 Fock matrices).
"""
from __future__ import annotations

import json
import os
import sys

CART = {L: [(x, y, L - x - y) for x in range(L, -1, -1) for y in range(L - x, -1, -1)] for L in range(9)}
PAIR_CLASSES = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2)]
PAIR_NAMES = ["ss", "ps", "pp", "ds", "dp", "dd"]
AX = "xyz"


def classes():
    out = []
    for X in range(len(PAIR_CLASSES)):
        for Y in range(X + 1):
            out.append((X, Y))
    return out


def cidx(t):
    return CART[sum(t)].index(t)


def tstr(t):
    return f"{sum(t)}_{cidx(t)}"


def sub(t, i, k=1):
    l = list(t)
    l[i] -= k
    return tuple(l)


def add(t, i, k=1):
    l = list(t)
    l[i] += k
    return tuple(l)


def first_nz(t):
    for i in range(3):
        if t[i] > 0:
            return i
    return -1


Z3 = (0, 0, 0)

# lanes that share one shell quartet's primitive work, by total angular momentum
LANES_BY_L = {0: 1, 1: 1, 2: 1, 3: 1, 4: 2, 5: 4, 6: 8, 7: 8, 8: 8}


class Counter:
    def __init__(self):
        self.prim = 0      # flops per primitive quartet (VRR + accumulation, excluding setup/Boys)
        self.cont = 0      # flops per contracted quartet (HRR + digestion)


def vname(e, f, m):
    return f"v{tstr(e)}_{tstr(f)}_{m}"


def all_targets(la, lb, lc, ld):
    """The contracted-quartet targets [e0|f0]^(0), l_a <= |e| <= l_a + l_b, l_c <= |f| <= l_c + l_d."""
    return [(e, f, 0) for le in range(la, la + lb + 1) for e in CART[le]
            for lf in range(lc, lc + ld + 1) for f in CART[lf]]


def gen_vrr(la, lb, lc, ld, cnt, subset=None):
    """Return (lines, accumulation lines, used coefficients, targets) for the VRR of one primitive quartet,
    restricted to the nodes the targets in `subset` (default: all) need."""
    L = la + lb + lc + ld
    targets = all_targets(la, lb, lc, ld) if subset is None else subset
    recipe = {}

    def need(node):
        if node in recipe:
            return
        e, f, m = node
        if e == Z3 and f == Z3:
            recipe[node] = ("base",)
            return
        if f == Z3:
            i = first_nz(e)
            e1 = sub(e, i)
            deps = [(e1, Z3, m), (e1, Z3, m + 1)]
            if e[i] >= 2:
                e2 = sub(e, i, 2)
                deps += [(e2, Z3, m), (e2, Z3, m + 1)]
            recipe[node] = ("e1", i, deps)
        else:
            i = first_nz(f)
            f1 = sub(f, i)
            deps = [(e, f1, m), (e, f1, m + 1)]
            if f[i] >= 2:
                f2 = sub(f, i, 2)
                deps += [(e, f2, m), (e, f2, m + 1)]
            if e[i] >= 1:
                deps += [(sub(e, i), f1, m + 1)]
            recipe[node] = ("e2", i, deps)
        for d in recipe[node][-1] if recipe[node][0] != "base" else []:
            need(d)

    for t in targets:
        need(t)
    order = sorted(recipe.keys(), key=lambda n: (sum(n[0]) + sum(n[1]), sum(n[1]), -n[2]))
    used = set()
    # WP_i = -(rho/p) PQ_i and WQ_i = (rho/q) PQ_i cost three multiplies per primitive quartet; when fewer
    # than three distinct values are multiplied by them, (rho/p) is folded into those values instead
    # (u = rho_p x, and WP_i x = -PQ_i u), which saves multiplies (the smallest classes only)
    wp_ops, wq_ops, wp_co, wq_co = set(), set(), set(), set()
    for node, r in recipe.items():
        if r[0] == "e1":
            wp_ops.add(vname(sub(node[0], r[1]), Z3, node[2] + 1))
            wp_co.add(r[1])
        elif r[0] == "e2":
            wq_ops.add(vname(node[0], sub(node[1], r[1]), node[2] + 1))
            wq_co.add(r[1])
    fold_p = FOLD and 0 < len(wp_ops) < len(wp_co)
    fold_q = FOLD and 0 < len(wq_ops) < len(wq_co)
    # the algorithmic count keeps the WP_i / WQ_i products (the setup counts them when they are formed)
    cnt.prim += (len(wp_co) if fold_p else 0) + (len(wq_co) if fold_q else 0)
    # targets no other node depends on are accumulated as an FMA chain of their recurrence terms
    # (acc = fma(c_k, x_k, acc) per term) instead of forming their value and adding it
    depended = set()
    for node, r in recipe.items():
        if r[0] != "base":
            depended.update(r[-1])
    tset = set(targets)
    leaf = {n for n in tset if n not in depended and recipe[n][0] != "base"}
    def fold_lines(nm):
        out_ = []
        if fold_p and nm in wp_ops:
            out_.append(f"const real up_{nm} = rho_p * {nm};")
        if fold_q and nm in wq_ops:
            out_.append(f"const real uq_{nm} = rho_q * {nm};")
        return out_

    lines = []
    acc = []
    for node in order:
        e, f, m = node
        r = recipe[node]
        nm = vname(e, f, m)
        if r[0] == "base":
            lines.append(f"const real {nm} = pref * F[{m}];")
            lines += fold_lines(nm)
            cnt.prim += 1
            continue
        i = r[1]
        a = AX[i]
        terms = []  # (coefficient, operand)
        if r[0] == "e1":
            e1 = sub(e, i)
            if fold_p:
                terms += [(f"PA{a}", vname(e1, Z3, m)), (f"-PQ{a}", "up_" + vname(e1, Z3, m + 1))]
                used.update({f"PA{a}", "rho_p"})
            else:
                terms += [(f"PA{a}", vname(e1, Z3, m)), (f"WP{a}", vname(e1, Z3, m + 1))]
                used.update({f"PA{a}", f"WP{a}"})
            cnt.prim += 3
            if e[i] >= 2:
                e2 = sub(e, i, 2)
                k = e[i] - 1
                terms.append((f"o2p_{k}", f"({vname(e2, Z3, m)} - rho_p * {vname(e2, Z3, m + 1)})"))
                used.update({f"o2p_{k}", "rho_p"})
                cnt.prim += 4
        else:
            f1 = sub(f, i)
            if fold_q:
                terms += [(f"QC{a}", vname(e, f1, m)), (f"PQ{a}", "uq_" + vname(e, f1, m + 1))]
                used.update({f"QC{a}", "rho_q"})
            else:
                terms += [(f"QC{a}", vname(e, f1, m)), (f"WQ{a}", vname(e, f1, m + 1))]
                used.update({f"QC{a}", f"WQ{a}"})
            cnt.prim += 3
            if f[i] >= 2:
                f2 = sub(f, i, 2)
                k = f[i] - 1
                terms.append((f"o2q_{k}", f"({vname(e, f2, m)} - rho_q * {vname(e, f2, m + 1)})"))
                used.update({f"o2q_{k}", "rho_q"})
                cnt.prim += 4
            if e[i] >= 1:
                k = e[i]
                terms.append((f"o2pq_{k}", vname(sub(e, i), f1, m + 1)))
                used.add(f"o2pq_{k}")
                cnt.prim += 2
        if node in leaf:
            an = f"acc{tstr(e)}_{tstr(f)}"
            for c, x in terms:
                lines.append(f"{an} = fma({c}, {x}, {an});")
        else:
            lines.append(f"const real {nm} = " + " + ".join(f"{c} * {x}" for c, x in terms) + ";")
        lines += fold_lines(nm)
    for (e, f, m) in targets:
        if (e, f, m) not in leaf:
            acc.append(f"acc{tstr(e)}_{tstr(f)} += {vname(e, f, 0)};")
        cnt.prim += 1
    return lines, acc, used, targets


RYS_MIN_L = 6  # classes that have a Rys-quadrature variant (all of them with HF_RYS)
# Classes whose FP64 launches use the Rys variant by default (neither HF_RYS nor HF_OBARA_SAIKA given): those
# where it measured faster than the Obara-Saika kernel on the 64-water build ((dd|pp) measured slower).
RYS_DEFAULT = {"2121", "2220", "2221", "2222"}
FOLD = True  # fold rho/p (rho/q) into the recurrence values when that saves multiplies


def gen_rys_prim(la, lb, lc, ld, cnt, subset=None):
    """Rys quadrature replacement of the vertical step for one primitive quartet: with the n = L/2 + 1
    nodes u_r = t_r^2 and weights w_r of the Boys weight at T (rys.cuh), and per node the 2D integrals
    G_d(a, c), d = x, y, z, a <= la + lb, c <= lc + ld, from
        G(0, 0) = 1 (x, y), pref w_r (z),
        G(a+1, 0) = C00 G(a, 0) + a B10 G(a-1, 0),
        G(a, c+1) = C00' G(a, c) + c B01 G(a, c-1) + a B00 G(a-1, c),
    with B00 = u / (2(p+q)), B10 = (1 - rho u / p) / (2p), B01 = (1 - rho u / q) / (2q),
    C00 = PA - (rho / p) u PQ, C00' = QC + (rho / q) u PQ (the Obara-Saika terms of the vertical
    recurrence with the m-th Boys value replaced by the m-th power of u), the targets are
    [e0|f0] += G_x(e_x, f_x) G_y(e_y, f_y) G_z(e_z, f_z), summed over the nodes.
    Returns (setup lines, per-primitive body lines, targets, setup flop count)."""
    L = la + lb + lc + ld
    n = L // 2 + 1
    targets = all_targets(la, lb, lc, ld) if subset is None else subset
    need = [set(), set(), set()]
    for e, f, _ in targets:
        for d in range(3):
            need[d].add((e[d], f[d]))
    # dependency closure in recurrence order
    for d in range(3):
        stack = list(need[d])
        while stack:
            a, c = stack.pop()
            deps = []
            if c > 0:
                deps = [(a, c - 1)] + ([(a, c - 2)] if c >= 2 else []) + ([(a - 1, c - 1)] if a >= 1 else [])
            elif a > 0:
                deps = [(a - 1, 0)] + ([(a - 2, 0)] if a >= 2 else [])
            for x in deps:
                if x not in need[d]:
                    need[d].add(x)
                    stack.append(x)
    setup = [
        "const real s = bp.p + kp.p;",
        "const real rs = rsq(s);",
        "const real inv = rs * rs;",
        "const real PQx = bp.Px - kp.Px, PQy = bp.Py - kp.Py, PQz = bp.Pz - kp.Pz;",
        "const real rho_p = kp.p * inv, rho_q = bp.p * inv, o2pq_1 = real(0.5) * inv, ko2p = kp.oo2p;",
        "const real rho = bp.p * rho_p;",
        "const real T = rho * (PQx * PQx + PQy * PQy + PQz * PQz);",
        "const real pref = bK * kp.K * rs;",
        "const real QCx = kp.PAx, QCy = kp.PAy, QCz = kp.PAz;",
        f"real ru[{n}], rw[{n}];",
        f"rys_rule<{n}>(T, ru, rw);",
    ]
    cset = 1 + 8 + 1 + 3 + 2 + 6 + 2 + 3 + 2 * n * 2 * 11 + 4
    body = [f"#pragma unroll 1", f"for (int r = 0; r < {n}; r++) {{",
            "    const real u = ru[r];",
            "    const real B00 = o2pq_1 * u;",
            "    const real B10 = bo2p - bo2p * rho_p * u;",
            "    const real B01 = ko2p - ko2p * rho_q * u;",
            "    const real up = rho_p * u, uq = rho_q * u;"]
    fl = 1 + 3 + 3 + 2
    for d, ax in enumerate(AX):
        body.append(f"    const real C{ax} = PA{ax} - up * PQ{ax}, D{ax} = QC{ax} + uq * PQ{ax};")
        fl += 4
    body.append("    const real gz_0_0 = pref * rw[r];")
    fl += 1
    for d, ax in enumerate(AX):
        g = f"g{ax}"
        nd = need[d]
        amax = max(a for a, c in nd)
        cmax = max(c for a, c in nd)
        for c in range(cmax + 1):
            for a in range(amax + 1):
                if (a, c) not in nd or (a, c) == (0, 0):
                    continue
                if c == 0:
                    expr = f"C{ax} * {g}_{a - 1}_0"
                    fl += 1
                    if a >= 2:
                        expr += f" + real({a - 1}) * B10 * {g}_{a - 2}_0"
                        fl += 3
                else:
                    expr = f"D{ax} * {g}_{a}_{c - 1}"
                    fl += 1
                    if c >= 2:
                        expr += f" + real({c - 1}) * B01 * {g}_{a}_{c - 2}"
                        fl += 3
                    if a >= 1:
                        expr += f" + real({a}) * B00 * {g}_{a - 1}_{c - 1}"
                        fl += 3
                body.append(f"    const real {g}_{a}_{c} = {expr};")
    for ax in "xy":
        body.insert(len(body) - sum(1 for _ in []), "")
    # G_x(0,0) = G_y(0,0) = 1: substitute the literal
    body = [l.replace("gx_0_0", "real(1)").replace("gy_0_0", "real(1)") for l in body if l != ""]
    for e, f, _ in targets:
        gx = f"gx_{e[0]}_{f[0]}" if (e[0], f[0]) != (0, 0) else None
        gy = f"gy_{e[1]}_{f[1]}" if (e[1], f[1]) != (0, 0) else None
        gz = f"gz_{e[2]}_{f[2]}"
        prod = " * ".join(x for x in (gx, gy, gz) if x)
        body.append(f"    acc{tstr(e)}_{tstr(f)} += {prod};")
        fl += 1 + (1 if gx else 0) + (1 if gy else 0)
    body.append("}")
    cnt.prim += fl * n
    return setup, body, targets, cset


def gen_setup(L, used, cnt):
    """Per-primitive-quartet quantities; returns lines (flop counts approximate the emitted ops)."""
    # rho = p q / (p + q) is formed as p (q / (p + q)) from rho_p where the recurrence needs rho_p anyway:
    # one FP64 multiply fewer per primitive quartet (the flop count keeps the two of the definition)
    lines = [
        "const real s = bp.p + kp.p;",
        "const real rs = rsq(s);",
        "const real inv = rs * rs;",
        "const real PQx = bp.Px - kp.Px, PQy = bp.Py - kp.Py, PQz = bp.Pz - kp.Pz;",
        "const real rho_p = kp.p * inv;" if L > 0 else "const real rho = bp.p * kp.p * inv;",
    ]
    if L > 0:
        lines += ["const real rho = bp.p * rho_p;"]
    lines += [
        "const real T = rho * (PQx * PQx + PQy * PQy + PQz * PQz);",
        "const real pref = bK * kp.K * rs;",
        f"real F[{L + 1}];",
        f"boys<real, {L}>(T, boys_tab, F);",
    ]
    cnt_setup = 1 + 8 + 1 + 3 + 2 + 6 + 2
    if L > 0:
        lines += ["const real rho_q = bp.p * inv;"]
        cnt_setup += 2
        for a in AX:
            if f"WP{a}" in used:
                lines.append(f"const real WP{a} = -rho_p * PQ{a};")
                cnt_setup += 1
            if f"WQ{a}" in used:
                lines.append(f"const real WQ{a} = rho_q * PQ{a};")
                cnt_setup += 1
        for k in range(1, 5):
            if f"o2p_{k}" in used:
                lines.append(f"const real o2p_{k} = real({k}) * bo2p;")
                cnt_setup += 1
            if f"o2q_{k}" in used:
                lines.append(f"const real o2q_{k} = real({k}) * kp.oo2p;")
                cnt_setup += 1
        if any(u.startswith("o2pq_") for u in used):
            lines.append("const real o2pq_1 = real(0.5) * inv;")
            cnt_setup += 1
            for k in range(2, 5):
                if f"o2pq_{k}" in used:
                    lines.append(f"const real o2pq_{k} = real({k}) * o2pq_1;")
                    cnt_setup += 1
        for a in AX:
            if f"QC{a}" in used:
                lines.append(f"const real QC{a} = kp.PA{a};")
    return lines, cnt_setup


def boys_flops(L):
    if L <= 1:
        return 5 + 7 * (L + 1) + 2
    return 5 + 7 + 9 + 1 + 2 * L + 2


def gen_hrr(la, lb, lc, ld, cnt):
    """HRR on the contracted [e0|f0]: returns lines and the name map of final x(a,b,c,d)."""
    lines = []
    fl = [f for lf in range(lc, lc + ld + 1) for f in CART[lf]]
    # bra: (a b| f) from (e 0| f)
    bra_name = {}

    def bname(a, b, f):
        return f"hb{tstr(a)}_{tstr(b)}_{tstr(f)}"

    for f in fl:
        memo = {}

        def need(a, b):
            if (a, b) in memo:
                return memo[(a, b)]
            if b == Z3:
                nm = f"acc{tstr(a)}_{tstr(f)}"
                memo[(a, b)] = nm
                return nm
            i = first_nz(b)
            n1 = need(add(a, i), sub(b, i))
            n2 = need(a, sub(b, i))
            nm = bname(a, b, f)
            lines.append(f"const real {nm} = {n1} + AB{AX[i]} * {n2};")
            cnt.cont += 2
            memo[(a, b)] = nm
            return nm

        for a in CART[la]:
            for b in CART[lb]:
                bra_name[(a, b, f)] = need(a, b)
    # ket: (a b| c d) from (a b| f 0)
    xname = {}
    for a in CART[la]:
        for b in CART[lb]:
            memo = {}

            def need2(c, d):
                if (c, d) in memo:
                    return memo[(c, d)]
                if d == Z3:
                    nm = bra_name[(a, b, c)]
                    memo[(c, d)] = nm
                    return nm
                i = first_nz(d)
                n1 = need2(add(c, i), sub(d, i))
                n2 = need2(c, sub(d, i))
                nm = f"hk{tstr(a)}_{tstr(b)}_{tstr(c)}_{tstr(d)}"
                lines.append(f"const real {nm} = {n1} + CD{AX[i]} * {n2};")
                cnt.cont += 2
                memo[(c, d)] = nm
                return nm

            for c in CART[lc]:
                for d in CART[ld]:
                    xname[(cidx(a), cidx(b), cidx(c), cidx(d))] = need2(c, d)
    return lines, xname


def gen_digest(la, lb, lc, ld, xname, cnt):
    na, nb, nc, nd = len(CART[la]), len(CART[lb]), len(CART[lc]), len(CART[ld])
    lines = []

    def x(a, b, c, d):
        return xname[(a, b, c, d)]

    def pload(tag, r0, n0, c0, n1):
        out = []
        for u in range(n0):
            for v in range(n1):
                out.append(f"const real P{tag}_{u}_{v} = (real)Pd[(size_t)({r0} + {u}) * N + {c0} + {v}];")
        return out

    # density blocks
    lines += pload("cd", "bC", nc, "bD", nd)
    lines += pload("ab", "bA", na, "bB", nb)
    lines += pload("bd", "bB", nb, "bD", nd)
    lines += pload("ac", "bA", na, "bC", nc)
    lines += pload("bc", "bB", nb, "bC", nc)
    lines += pload("ad", "bA", na, "bD", nd)

    def block(target, r0, n0, c0, n1, terms, scale):
        for u in range(n0):
            for v in range(n1):
                ts = terms(u, v)
                expr = " + ".join(f"{xx} * {pp}" for xx, pp in ts)
                cnt.cont += 2 * len(ts) + 1
                lines.append(f"red_add(&{target}[(size_t)({r0} + {u}) * N + {c0} + {v}], (double)({scale} * ({expr})));")

    block("Jt", "bA", na, "bB", nb, lambda a, b: [(x(a, b, c, d), f"Pcd_{c}_{d}") for c in range(nc) for d in range(nd)], "fj")
    block("Jt", "bC", nc, "bD", nd, lambda c, d: [(x(a, b, c, d), f"Pab_{a}_{b}") for a in range(na) for b in range(nb)], "fj")
    block("Kt", "bA", na, "bC", nc, lambda a, c: [(x(a, b, c, d), f"Pbd_{b}_{d}") for b in range(nb) for d in range(nd)], "fk")
    block("Kt", "bB", nb, "bD", nd, lambda b, d: [(x(a, b, c, d), f"Pac_{a}_{c}") for a in range(na) for c in range(nc)], "fk")
    block("Kt", "bA", na, "bD", nd, lambda a, d: [(x(a, b, c, d), f"Pbc_{b}_{c}") for b in range(nb) for c in range(nc)], "fk")
    block("Kt", "bB", nb, "bC", nc, lambda b, c: [(x(a, b, c, d), f"Pad_{a}_{d}") for a in range(na) for d in range(nd)], "fk")
    return lines


def gen_schwarz(la, lb, xname):
    """max over (a,b) of |(ab|ab)| times the component-normalisation factors."""
    na, nb = len(CART[la]), len(CART[lb])
    lines = ["double qmax = 0.0;"]
    for a in range(na):
        for b in range(nb):
            na_ = comp_norm2(CART[la][a]) * comp_norm2(CART[lb][b])
            lines.append(f"qmax = fmax(qmax, fabs((double){xname[(a, b, a, b)]}) * {na_!r});")
    return lines


def comp_norm2(t):
    """Square of the Cartesian component factor 1/sqrt((2i-1)!!(2j-1)!!(2k-1)!!)."""
    def df(n):
        r = 1
        while n > 1:
            r *= n
            n -= 2
        return r
    return 1.0 / (df(2 * t[0] - 1) * df(2 * t[1] - 1) * df(2 * t[2] - 1))


def class_name(X, Y):
    la, lb = PAIR_CLASSES[X]
    lc, ld = PAIR_CLASSES[Y]
    return f"{la}{lb}{lc}{ld}"


# Largest number of accumulators per pass over the primitives, by sizeof(real).  FP32 classes with more
# targets run in passes (measured: (dd|dp) 43 -> 10.5 ms, (dd|dd) 15 -> 10 ms at 64 waters); the FP64
# kernels, bound by the FP64 pipe, lost more to the repeated setup than they gained from fewer spills
# ((dp|dp) +17%, (dd|dd) +42%), so they run in one pass.
CHUNK = {8: 10 ** 9, 4: 192}


def target_chunks(targets, size):
    """Consecutive chunks (targets are ordered by bra component, so a chunk shares its bra recurrence)."""
    return [targets[i:i + size] for i in range(0, len(targets), size)]


def gen_class(X, Y, method="os"):
    """Source of one class's quartet function and kernels: method "os" (Obara-Saika vertical step, Boys
    table) or "rys" (Rys quadrature vertical step); both share the contraction, HRR and digestion.

    A class with more targets than fit in registers (CHUNK, per arithmetic type) runs its primitive loop
    in passes, each accumulating one chunk of targets with only the recurrence nodes that chunk needs; the
    finished chunks are kept in a per-thread array for the horizontal step.  The reported flop counts are
    those of a single pass over every target (the algorithm's work, not the repeated setup)."""
    la, lb = PAIR_CLASSES[X]
    lc, ld = PAIR_CLASSES[Y]
    L = la + lb + lc + ld
    name = class_name(X, Y)
    cnt = Counter()
    if method == "os":
        vrr, acc, used, targets = gen_vrr(la, lb, lc, ld, cnt)
        setup, cset = gen_setup(L, used, cnt)
        extra = boys_flops(L)
        qname = f"quartet_{name}"
    else:
        setup, vrr, targets, cset = gen_rys_prim(la, lb, lc, ld, cnt)
        acc = []
        used = {"PAx", "PAy", "PAz"}
        extra = 0
        qname = f"quartet_rys_{name}"
    hrr, xname = gen_hrr(la, lb, lc, ld, cnt)
    cont_hrr = cnt.cont
    dig = gen_digest(la, lb, lc, ld, xname, cnt)
    prim_flops = cnt.prim + cset + extra
    tnames = [f"acc{tstr(e)}_{tstr(f)}" for (e, f, m) in targets]
    need_ab = any("AB" in l for l in hrr)
    need_cd = any("CD" in l for l in hrr)
    G = LANES_BY_L[L]

    def prim_body(chunk):
        """Lines of one primitive quartet for the targets of `chunk`."""
        c2 = Counter()
        if method == "os":
            v, a_, u, _ = gen_vrr(la, lb, lc, ld, c2, chunk)
            st, _ = gen_setup(L, u, c2)
        else:
            st, v, _, _ = gen_rys_prim(la, lb, lc, ld, c2, chunk)
            a_, u = [], {"PAx", "PAy", "PAz"}
        lines = ["const real bK = bp.K, bo2p = bp.oo2p;"]
        lines += [f"const real PA{x} = bp.PA{x};" for x in AX if f"PA{x}" in u]
        lines += st
        # each target is accumulated right after its recurrence node, which keeps fewer values alive
        acc_of = {l.split(" += ")[1].rstrip(";"): l for l in a_}
        for l in v:
            lines.append(l)
            if l.startswith("const real v"):
                nm = l.split(" = ")[0].split()[-1]
                if nm in acc_of:
                    lines.append(acc_of.pop(nm))
        lines += list(acc_of.values())
        return lines

    def loop_lines(chunk, first, order):
        """The loop over the primitive staircase for `chunk`: order "bra" (bra-major, the FP64 kernels) or
        "ket" (ket-major, the FP32 kernels: a lane reloads its ket record only when its ket primitive
        changes, which removes most of the ket loads that bound them on L1)."""
        o = ["// lane l evaluates staircase positions l, l + G, l + 2G, ... in lockstep with its group"]
        if order == "bra":
            o += ["int nkb = nkb0, ib = 0, ik = 0;",
                  "auto advance = [&]() {",
                  "    if (++ik == nkb) {",
                  "        ik = 0;",
                  "        ib++;",
                  "        if (ib < nbp)",
                  "            while (nkb > 0 && bpp[ib].B * kv.B(nkb - 1) < ptau) nkb--;",
                  "    }",
                  "};"]
        else:
            o += ["int nbb = nbb0, ib = 0, ik = 0, lk = -1;",
                  "PrimPair<real> kp;",
                  "auto advance = [&]() {",
                  "    if (++ib == nbb) {",
                  "        ib = 0;",
                  "        ik++;",
                  "        if (ik < nkp)",
                  "            while (nbb > 0 && bpp[nbb - 1].B * kv.B(ik) < ptau) nbb--;",
                  "    }",
                  "};"]
        o += ["if (G > 1)",
              "    for (int s = 0; s < lane && s < total; s++) advance();",
              "for (int it = (G > 1 ? lane : 0); it < total; it += G) {",
              "    const int cib = ib, cik = ik;",
              "#pragma unroll",
              "    for (int s = 0; s < G; s++) advance();"]
        if first:
            o.append("    nq++;")
        o.append("    const PrimPair<real> bp = bpp[cib];")
        if order == "bra":
            o.append("    const PrimPair<real> kp = kv.rec(cik);")
        else:
            o += ["    if (cik != lk) {", "        kp = kv.rec(cik);", "        lk = cik;", "    }"]
        o += ["    " + l for l in prim_body(chunk)]
        o.append("}")
        return o

    def shuffle_lines(chunk):
        cn = [f"acc{tstr(e)}_{tstr(f)}" for (e, f, m) in chunk]
        o = ["if constexpr (G > 1) {", "#pragma unroll", "    for (int o = 1; o < G; o <<= 1) {"]
        o += [f"        {nm} += __shfl_xor_sync(0xffffffffu, {nm}, o);" for nm in cn]
        o += ["    }", "}"]
        return o

    def pass_lines(chunk, first, store, order):
        """One pass over the primitive staircase accumulating `chunk` (its own scope)."""
        cn = [f"acc{tstr(e)}_{tstr(f)}" for (e, f, m) in chunk]
        o = ["{"]
        o += [f"    real {nm} = real(0);" for nm in cn]
        o += ["    " + l for l in loop_lines(chunk, first, order)]
        o += ["    " + l for l in shuffle_lines(chunk)]
        if store:
            o += [f"    accv[{tnames.index(nm)}] = {nm};" for nm in cn]
        o.append("}")
        return o

    ch = {sz: target_chunks(targets, CHUNK[sz]) for sz in (8, 4)}
    chunked = len(ch[8]) > 1 or len(ch[4]) > 1

    out = []
    out.append(f"// ({PAIR_NAMES[X]}|{PAIR_NAMES[Y]}) class: l = {la}{lb}{lc}{ld}, "
               f"{len(targets)} [e0|f0] targets, {prim_flops} flops per primitive quartet, "
               f"{cnt.cont} per contracted quartet" + (", Rys quadrature" if method == "rys" else "")
               + (f"; {len(ch[8])} passes in FP64, {len(ch[4])} in FP32." if chunked else "."))
    out.append(f"// Lanes per quartet in the ERI kernels: {G}.  The G lanes of a group share one shell quartet's")
    out.append(f"// primitive staircase round-robin and sum their accumulators with butterfly shuffles; lane 0")
    out.append(f"// then runs the horizontal recurrence and the digestion.  Called warp-uniformly; a lane with")
    out.append(f"// valid == false takes part in the shuffles only.")
    out.append(f"template <typename real, int G, typename KV>")
    out.append(f"__device__ __forceinline__ int {qname}(const PairHdr& hb, const PairHdr& hk, const KV& kv,"
               f" const PrimPair<real>* __restrict__ prims, const real* __restrict__ boys_tab,")
    out.append(f"    const real* __restrict__ Pd, int N, real fscale, double* __restrict__ Jt, double* __restrict__ Kt, double* qout,")
    out.append(f"    float ptau, int lane, bool valid)")
    out.append("{")
    out.append("    // surviving primitive quartets form a staircase (pairs sorted by bound): bra primitive ib pairs")
    out.append("    // with the first nk(ib) ket primitives, nk non-increasing (equivalently ket primitive ik with the")
    out.append("    // first nb(ik) bra primitives); one flat loop over it, bra-major in FP64, ket-major in FP32.")
    out.append("    // kv: the ket's records (KetAos: the pair's record array; KetSoa: its column of the class's ket table)")
    out.append("    const PrimPair<real>* __restrict__ bpp = prims + hb.prim0;")
    out.append("    const int nbp = hb.nprim, nkp = hk.nprim;")
    out.append("    int nkb0 = nkp, nbb0 = nbp;")
    out.append("    int total = 0;")
    out.append("    if (valid) {")
    out.append("        for (int ib = 0, c = nkb0; ib < nbp; ib++) {")
    out.append("            const float Bb = bpp[ib].B;")
    out.append("            while (c > 0 && Bb * kv.B(c - 1) < ptau) c--;")
    out.append("            if (c == 0) break;")
    out.append("            total += c;")
    out.append("        }")
    out.append("        while (nkb0 > 0 && bpp[0].B * kv.B(nkb0 - 1) < ptau) nkb0--;")
    out.append("        while (nbb0 > 0 && bpp[nbb0 - 1].B * kv.B(0) < ptau) nbb0--;")
    out.append("    }")
    out.append("    int nq = 0;")
    if not chunked:
        # single pass: the accumulators stay in scope for the horizontal step
        out += [f"    real {nm} = real(0);" for nm in tnames]
        out.append("    if constexpr (sizeof(real) == 8) {")
        out += ["        " + l for l in loop_lines(targets, True, "bra")]
        out.append("    } else {")
        out += ["        " + l for l in loop_lines(targets, True, "ket")]
        out.append("    }")
        out += ["    " + l for l in shuffle_lines(targets)]
    else:
        out.append(f"    real accv[{len(targets)}];  // finished chunks of targets")
        for sz, kw in ((8, "if constexpr (sizeof(real) == 8)"), (4, "else")):
            out.append(f"    {kw} {{")
            for k, c in enumerate(ch[sz]):
                out += ["        " + l for l in pass_lines(c, k == 0, True, "bra" if sz == 8 else "ket")]
            out.append("    }")
        out += [f"    const real {nm} = accv[{i}];" for i, nm in enumerate(tnames)]
    out.append("    if (!valid || lane != 0) return nq;")
    tail = []
    if need_ab:
        tail.append("const real ABx = pair_ab<real>(hb.ABx, hb.ABfx), ABy = pair_ab<real>(hb.ABy, hb.ABfy), "
                    "ABz = pair_ab<real>(hb.ABz, hb.ABfz);")
    if need_cd:
        tail.append("const real CDx = pair_ab<real>(hk.ABx, hk.ABfx), CDy = pair_ab<real>(hk.ABy, hk.ABfy), "
                    "CDz = pair_ab<real>(hk.ABz, hk.ABfz);")
    tail += hrr
    tail.append("if (qout) {")
    if X == Y:
        tail += ["    " + l for l in gen_schwarz(la, lb, xname)]
        tail.append("    *qout = qmax;")
    tail.append("    return;")
    tail.append("}")
    tail.append("if (total == 0) return;  // every primitive quartet screened: nothing to digest")
    tail.append("const int bA = hb.bfA, bB = hb.bfB, bC = hk.bfA, bD = hk.bfB;")
    tail.append("const real fj = real(4) * fscale, fk = real(2) * fscale;")
    tail += dig
    out += ["    " + l.replace("return;", "return nq;") for l in tail]
    out.append("    return nq;")
    out.append("}")
    out.append("")
    if method == "rys":
        out.append(f"ERI_RYS_KERNELS({name}, {G})")
    else:
        out.append(f"ERI_BATCH_KERNEL({name}, {G})")
        out.append(f"ERI_CLASS_KERNELS({name}, {X}, {Y}, {G})")
        if X == Y:
            out.append(f"SCHWARZ_KERNEL({name})")
    info = dict(name=name, X=X, Y=Y, l=[la, lb, lc, ld], L=L, G=G, prim_flops=prim_flops, cont_flops=cnt.cont,
                hrr_flops=cont_hrr, targets=len(targets), vrr_nodes=len(vrr))
    return "\n".join(out) + "\n", info


HEADER = """// Generated by gen_eri.py: do not edit.  One shell-quartet class per file.
#include "eri_common.cuh"

namespace hf {
"""
FOOTER = "}  // namespace hf\n"


def main(outdir):
    os.makedirs(outdir, exist_ok=True)
    infos = []
    for X, Y in classes():
        src, info = gen_class(X, Y)
        infos.append(info)
        path = os.path.join(outdir, f"eri_{info['name']}.cu")
        text = HEADER + src + FOOTER
        if not os.path.exists(path) or open(path).read() != text:
            with open(path, "w") as fh:
                fh.write(text)
        info["rys"] = info["L"] >= RYS_MIN_L
        info["prim_flops_rys"] = 0
        if info["rys"]:
            rsrc, rinfo = gen_class(X, Y, "rys")
            info["prim_flops_rys"] = rinfo["prim_flops"]
            path = os.path.join(outdir, f"eri_rys_{info['name']}.cu")
            text = HEADER.replace('#include "eri_common.cuh"', '#include "eri_common.cuh"\n#include "rys.cuh"') + rsrc + FOOTER
            if not os.path.exists(path) or open(path).read() != text:
                with open(path, "w") as fh:
                    fh.write(text)
    # dispatch table
    lines = ['// Generated by gen_eri.py: do not edit.', '#include "eri_common.cuh"', "", "namespace hf {"]
    for info in infos:
        n = info["name"]
        lines.append(f"void launch_eri_{n}(const EriArgs&, int, int, int, cudaStream_t, int);")
        if info["X"] == info["Y"]:
            lines.append(f"void launch_schwarz_{n}(const SchwarzArgs&, int, cudaStream_t);")
        lines.append(f"void launch_eri_batch_{n}(const BatchArgs&, int, int, cudaStream_t);")
        lines.append(f"size_t local_bytes_{n}();")
        if info["rys"]:
            lines.append(f"void launch_eri_rys_{n}(const EriArgs&, int, int, int, cudaStream_t, int);")
            lines.append(f"size_t local_bytes_rys_{n}();")
    lines.append("")
    lines.append("const EriClassEntry kEriClasses[kNumClasses] = {")
    for info in infos:
        n = info["name"]
        lines.append(f"    {{{info['X']}, {info['Y']}, {info['L']}, {info['prim_flops']}, {info['cont_flops']}, "
                     f"launch_eri_{n}, {('launch_schwarz_' + n) if info['X'] == info['Y'] else 'nullptr'}, \"{n}\", "
                     f"launch_eri_batch_{n}, local_bytes_{n}, {info['G']}, "
                     + (f"launch_eri_rys_{n}, {info['prim_flops_rys']}, local_bytes_rys_{n}, "
                        f"{1 if n in RYS_DEFAULT else 0}}}," if info["rys"]
                        else "nullptr, 0, nullptr, 0},"))
    lines.append("};")
    lines.append("}  // namespace hf")
    text = "\n".join(lines) + "\n"
    path = os.path.join(outdir, "eri_table.cu")
    if not os.path.exists(path) or open(path).read() != text:
        with open(path, "w") as fh:
            fh.write(text)
    jpath = os.path.join(outdir, "eri_classes.json")
    with open(jpath, "w") as fh:
        json.dump(infos, fh, indent=1)
    return infos


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser(description="Generate the per-class ERI kernels and their table.")
    ap.add_argument("out", nargs="?", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "generated"),
                    help="output directory (default: the package's csrc/generated)")
    main(ap.parse_args().out)
