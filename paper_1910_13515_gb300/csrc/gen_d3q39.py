#!/usr/bin/env python3
"""Generate d3q39_gen.cuh: straight-line D3Q39 arithmetic for the CUDA kernels.

Run from this directory: ``python gen_d3q39.py`` (the output is committed; the build does
not run this script).

The 39 velocities split into sign orbits: all velocities with the same |xi_x|, |xi_y|,
|xi_z| (13 orbits of size 1, 2, 4 or 8).  On an orbit with non-zero axes S and magnitudes
a, a monomial xi^p equals prod_a a^p * prod_{p_a odd} s_a, so
  * a moment sum_i F_i xi_i^p is a sum over orbits of an integer times one Walsh-Hadamard
    coefficient H_T = sum_s F(s) prod_{a in T} s_a (T = axes with odd power);
  * the exponent sum_k lam_k phi_k(xi) on an orbit is sum_T c_T prod_{a in T} s_a, whose 2^|S|
    values follow from the coefficients c_T by the same butterflies.
This is the same arithmetic as the plain sums over 39 velocities, reorganised.

Emitted:
  exponents<T>(l, e)          e_i = sum_k l_k phi_k(xi_i)         (Eq. discrete-equilibrium)
  moments<T>(F, s, J)         s_k = sum_i F_i phi_k,  J_kl = sum_i F_i phi_k phi_l (packed)
  f_moments(f, ...)           rho, j, sum f|xi|^2;  g_sum(g): sum g
  exp2_table                  2^(j/256), j = 0..255, correctly rounded (decimal arithmetic)
  exp constants               ln2/256 split in a 32-bit head and a tail
"""
from __future__ import annotations

import decimal
import itertools
import os
from collections import defaultdict

D = decimal.Decimal
decimal.getcontext().prec = 60

HERE = os.path.dirname(os.path.abspath(__file__))

CX = [0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, -1, 1, 2, -2, 0, 0, 0,
      0, 2, -2, 2, -2, 2, -2, 2, -2, 0, 0, 0, 0, 3, -3, 0, 0, 0, 0]
CY = [0, 0, 0, 1, -1, 0, 0, 1, -1, 1, -1, -1, 1, 1, -1, 0, 0, 2, -2, 0,
      0, 2, -2, -2, 2, 0, 0, 0, 0, 2, -2, 2, -2, 0, 0, 3, -3, 0, 0]
CZ = [0, 0, 0, 0, 0, 1, -1, 1, -1, -1, 1, 1, -1, 1, -1, 0, 0, 0, 0, 2,
      -2, 0, 0, 0, 0, 2, -2, -2, 2, 2, -2, -2, 2, 0, 0, 0, 0, 3, -3]
Q = 39
VEL = [(CX[i], CY[i], CZ[i]) for i in range(Q)]
NM = 13
# basis exponents (p, q, r) of phi_k, with |xi|^2 expanded: phi_10..12 are sums of monomials
BASIS = [
    {(0, 0, 0): 1},
    {(1, 0, 0): 1}, {(0, 1, 0): 1}, {(0, 0, 1): 1},
    {(2, 0, 0): 1}, {(0, 2, 0): 1}, {(0, 0, 2): 1},
    {(1, 1, 0): 1}, {(1, 0, 1): 1}, {(0, 1, 1): 1},
    {(3, 0, 0): 1, (1, 2, 0): 1, (1, 0, 2): 1},
    {(2, 1, 0): 1, (0, 3, 0): 1, (0, 1, 2): 1},
    {(2, 0, 1): 1, (0, 2, 1): 1, (0, 0, 3): 1},
]


def tri(k, l):
    return k * (k + 1) // 2 + l


def phi(k, v):
    return sum(c * v[0] ** p * v[1] ** q * v[2] ** r for (p, q, r), c in BASIS[k].items())


# ---------------------------------------------------------------------------------------
# Orbits: key = (|x|, |y|, |z|); members listed with their sign tuple.

def orbits():
    orb = defaultdict(list)
    for i, v in enumerate(VEL):
        orb[tuple(abs(c) for c in v)].append(i)
    out = []
    for key in sorted(orb):
        axes = [a for a in range(3) if key[a] != 0]
        members = {}
        for i in orb[key]:
            s = tuple(1 if VEL[i][a] > 0 else -1 for a in axes)
            members[s] = i
        out.append((key, axes, members))
    return out


ORBITS = orbits()
assert sum(len(m) for _, _, m in ORBITS) == Q


def subsets(axes):
    for r in range(len(axes) + 1):
        for T in itertools.combinations(axes, r):
            yield T


def hname(o, T):
    key = ORBITS[o][0]
    return "h%d%d%d_%s" % (key + ("".join("xyz"[a] for a in T) or "0",))


class Emitter:
    def __init__(self):
        self.lines = []

    def __call__(self, s):
        self.lines.append(s)


def tree_sum(names):
    """Balanced parenthesised sum (dependency depth log2 n instead of n)."""
    if len(names) == 1:
        return names[0]
    h = (len(names) + 1) // 2
    return f"({tree_sum(names[:h])} + {tree_sum(names[h:])})"


def lincomb(terms, T="T"):
    """Expression for sum c*v with integer c (no multiply by 1): for more than 4 terms, up to
    4 independent FMA/ADD chains, each headed by a coefficient +-1 term where there is one,
    added pairwise -- the same operation count as one chain, a quarter of its depth."""
    terms = [(c, v) for c, v in terms if c != 0]
    if not terms:
        return "T(0)".replace("T", T)
    if len(terms) > 4:
        k = 2 if len(terms) <= 8 else 4
        ones = [t for t in terms if t[0] == 1] + [t for t in terms if t[0] == -1]
        rest = [t for t in terms if abs(t[0]) != 1]
        heads = ones[:k]
        pool = ones[k:] + rest
        groups = [[h] for h in heads] + [[] for _ in range(k - len(heads))]
        for j, t in enumerate(pool):
            groups[j % k].append(t)
        groups = [g for g in groups if g]
        return tree_sum([f"({lincomb_chain(g, T)})" for g in groups])
    return lincomb_chain(terms, T)


def lincomb_chain(terms, T):
    """One FMA/ADD chain for sum c*v."""
    terms = list(terms)
    # start with a coefficient-1 term if any
    terms.sort(key=lambda cv: (abs(cv[0]) != 1, cv[0] < 0))
    c, v = terms[0]
    if c == 1:
        e = v
    elif c == -1:
        e = f"-{v}"
    else:
        # a product that the compiler may not fuse into a later add: the rounding of every
        # sum is then fixed by this text, whatever other uses of the product remain
        e = f"mul_rn({T}({c}), {v})"
    for c, v in terms[1:]:
        if c == 1:
            e = f"{e} + {v}"
        elif c == -1:
            e = f"{e} - {v}"
        else:
            e = f"fma({T}({c}), {v}, {e})"
    return e


def gen_fold(em, T):
    """F (39 values, array F) -> Walsh-Hadamard coefficients of every orbit."""
    for o, (key, axes, members) in enumerate(ORBITS):
        n = len(axes)
        # current stage values: dict from (sign tuple prefix-transformed) -> expr name
        cur = {s: f"F[{i}]" for s, i in members.items()}
        # transform axis by axis: after transforming axis a, index position a holds
        # '+' (sum) or '*' (difference, i.e. odd in that axis)
        for stage, a in enumerate(axes):
            nxt = {}
            for s in cur:
                if s[stage] == 1:
                    sm = s[:stage] + (-1,) + s[stage + 1:]
                    n_even = s[:stage] + ("E",) + s[stage + 1:]
                    n_odd = s[:stage] + ("O",) + s[stage + 1:]
                    ve = f"w{o}_{stage}_{len(nxt)}"
                    vo = f"w{o}_{stage}_{len(nxt) + 1}"
                    em(f"  const {T} {ve} = {cur[s]} + {cur[sm]};")
                    em(f"  const {T} {vo} = {cur[s]} - {cur[sm]};")
                    nxt[n_even] = ve
                    nxt[n_odd] = vo
            cur = nxt
        for s, v in cur.items():
            Tset = tuple(axes[j] for j in range(n) if s[j] == "O")
            em(f"  const {T} {hname(o, Tset)} = {v};")


# phi_k = |xi|^(2 m_k) xi^(p_k): (p_k, m_k); |xi|^2 is constant on an orbit
GBASIS = [((0, 0, 0), 0), ((1, 0, 0), 0), ((0, 1, 0), 0), ((0, 0, 1), 0), ((2, 0, 0), 0),
          ((0, 2, 0), 0), ((0, 0, 2), 0), ((1, 1, 0), 0), ((1, 0, 1), 0), ((0, 1, 1), 0),
          ((1, 0, 0), 1), ((0, 1, 0), 1), ((0, 0, 1), 1)]


# basis functions even in xi_z: on a lattice one cell thick in z whose populations are
# mirror-symmetric in z (u_z = 0), the other four multipliers stay exactly zero and their
# rows of J are exact zeros off the diagonal block, so the solve reduces to these nine.
ZEVEN = [k for k in range(NM) if GBASIS[k][0][2] % 2 == 0]
assert ZEVEN == [0, 1, 2, 4, 5, 6, 7, 10, 11]
N2 = len(ZEVEN)


def monomial_moment_terms(p, m=0):
    """sum_i F_i |xi_i|^(2m) xi_i^p as integer * Walsh coefficient terms."""
    terms = []
    for o, (key, axes, members) in enumerate(ORBITS):
        if any(p[a] != 0 and key[a] == 0 for a in range(3)):
            continue
        mag = sum(k * k for k in key) ** m
        for a in range(3):
            mag *= key[a] ** p[a]
        if mag == 0:
            continue
        Tset = tuple(a for a in axes if p[a] % 2 == 1)
        terms.append((mag, hname(o, Tset)))
    return terms


def gen_moments():
    em = Emitter()
    em("// s_k = sum_i F_i phi_k(xi_i) and J_kl = sum_i F_i phi_k(xi_i) phi_l(xi_i) (l <= k,")
    em("// packed) from the Walsh-Hadamard coefficients of the sign orbits.")
    em("template <class T, class A>")
    em("__device__ __forceinline__ void moments(const A& F, T (&s)[13], T (&J)[91]) {")
    gen_fold(em, "T")
    # distinct generalised monomials |xi|^(2m) xi^p needed by s and J
    need = {}
    for k in range(NM):
        need[GBASIS[k]] = None
        for l in range(k + 1):
            pk, mk = GBASIS[k]
            pl, ml = GBASIS[l]
            need[(tuple(a + b for a, b in zip(pk, pl)), mk + ml)] = None
    monos = sorted(need, key=lambda pm: (pm[1], sum(pm[0]), pm[0]))
    names = {}
    for (p, m) in monos:
        nm = "M%d%d%d_%d" % (p + (m,))
        names[(p, m)] = nm
        em(f"  const T {nm} = {lincomb(monomial_moment_terms(p, m), 'T')};")
    for k in range(NM):
        em(f"  s[{k}] = {names[GBASIS[k]]};")
    body_s = [ln for ln in em.lines]
    for k in range(NM):
        for l in range(k + 1):
            pk, mk = GBASIS[k]
            pl, ml = GBASIS[l]
            em(f"  J[{tri(k, l)}] = {names[(tuple(a + b for a, b in zip(pk, pl)), mk + ml)]};")
    em("}")
    # residual-only variant: the same fold and the 13 basis moments (unused values are dead code)
    only = ["", "// s_k = sum_i F_i phi_k(xi_i) only.", "template <class T, class A>",
            "__device__ __forceinline__ void moments_s(const A& F, T (&s)[13]) {"]
    keep = {names[GBASIS[k]] for k in range(NM)}
    for ln in body_s[4:]:
        if ln.lstrip().startswith("const T M") and ln.split()[2] not in keep:
            continue
        only.append(ln)
    only.append("}")
    # z-mirror variants (9 z-even basis functions): the same fold and the same monomial
    # expressions, restricted to what the z-even s and J need (the rest is dead code)
    def two_d(signature, with_J):
        out = ["", signature]
        keep2 = {names[GBASIS[k]] for k in ZEVEN}
        if with_J:
            for a, k in enumerate(ZEVEN):
                for b, l in enumerate(ZEVEN[:a + 1]):
                    pk, mk = GBASIS[k]
                    pl, ml = GBASIS[l]
                    keep2.add(names[(tuple(x + y for x, y in zip(pk, pl)), mk + ml)])
        for ln in body_s[4:]:
            if ln.lstrip().startswith("s["):
                continue
            if ln.lstrip().startswith("const T M") and ln.split()[2] not in keep2:
                continue
            out.append(ln)
        for a, k in enumerate(ZEVEN):
            out.append(f"  s[{a}] = {names[GBASIS[k]]};")
        if with_J:
            for a, k in enumerate(ZEVEN):
                for b, l in enumerate(ZEVEN[:a + 1]):
                    pk, mk = GBASIS[k]
                    pl, ml = GBASIS[l]
                    out.append(f"  J[{tri(a, b)}] = "
                               f"{names[(tuple(x + y for x, y in zip(pk, pl)), mk + ml)]};")
        out.append("}")
        return out
    d2 = (["", "// z-mirror-symmetric F: s and J of the nine z-even basis functions (ZEVEN order)."]
          + ["template <class T, class A>"]
          + two_d("__device__ __forceinline__ void moments2d(const A& F, T (&s)[9], T (&J)[45]) {",
                  True)[1:]
          + ["", "template <class T, class A>"]
          + two_d("__device__ __forceinline__ void moments_s2d(const A& F, T (&s)[9]) {",
                  False)[1:])
    return em.lines + only + d2, len(monos)


def gen_exponents(zsym=False):
    """e_i = sum_k l_k phi_k(xi_i) for the 39 velocities, per orbit: the coefficients c_T of
    the sign monomials, then the inverse butterflies.  zsym: the z-odd multipliers are zero
    (not read); z-mirrored velocities get the same exponent expression."""
    em = Emitter()
    if zsym:
        em("// The same with the z-odd multipliers zero (lattice one cell thick in z, u_z = 0).")
        em("template <class T>")
        em("__device__ __forceinline__ void exponents2d(const T (&l)[13], T (&e)[39]) {")
    else:
        em("// e_i = sum_k l_k phi_k(xi_i) for every velocity (exponent of Eq. discrete-equilibrium),")
        em("// in the type of l (double; float for the single-precision start of a solve).")
        em("template <class T>")
        em("__device__ __forceinline__ void exponents(const T (&l)[13], T (&e)[39]) {")
    for o, (key, axes, members) in enumerate(ORBITS):
        n = len(axes)
        # c_T = sum_k l_k * (coefficient of prod_{a in T} s_a in phi_k on this orbit)
        cT = {}
        for Tset in subsets(axes):
            terms = []
            for k in range(NM):
                if zsym and k not in ZEVEN:
                    continue
                coef = 0
                for p, c in BASIS[k].items():
                    if any(p[a] != 0 and key[a] == 0 for a in range(3)):
                        continue
                    odd = tuple(a for a in axes if p[a] % 2 == 1)
                    if odd != Tset:
                        continue
                    mag = c
                    for a in range(3):
                        mag *= key[a] ** p[a]
                    coef += mag
                if coef:
                    terms.append((coef, f"l[{k}]"))
            cT[Tset] = terms
        # emit coefficients
        cname = {}
        for Tset, terms in cT.items():
            nm = "c%d_%s" % (o, "".join("xyz"[a] for a in Tset) or "0")
            if terms:
                em(f"  const T {nm} = {lincomb(terms, 'T')};")
                cname[Tset] = nm
            else:
                cname[Tset] = None
        # inverse transform: value(s) = sum_T c_T prod_{a in T} s_a, built axis by axis
        # start: dict over partial sign assignment of the first j axes -> dict T-> expr
        # simple approach: for each s, accumulate with butterflies over subsets
        # stage form: v[(signs for processed axes), (remaining subset)]
        cur = {((), Tset): cname[Tset] for Tset in cT}
        for j, a in enumerate(axes):
            nxt = {}
            for (sg, Tset), v in cur.items():
                if a in Tset:
                    continue
                T_with = tuple(sorted(Tset + (a,)))
                vo = cur.get((sg, T_with))
                for sa in (1, -1):
                    key2 = (sg + (sa,), Tset)
                    if v is None and vo is None:
                        nxt[key2] = None
                        continue
                    nm = f"t{o}_{j}_{len(nxt)}"
                    if vo is None:
                        expr = v
                    elif v is None:
                        expr = vo if sa == 1 else f"-{vo}"
                    else:
                        expr = f"{v} + {vo}" if sa == 1 else f"{v} - {vo}"
                    if expr == v or expr == vo:
                        nxt[key2] = expr
                    else:
                        em(f"  const T {nm} = {expr};")
                        nxt[key2] = nm
            cur = nxt
        for (sg, Tset), v in cur.items():
            assert Tset == ()
            i = members[sg]
            em(f"  e[{i}] = {v if v is not None else 'T(0)'};")
    em("}")
    return em.lines


def gen_pop_moments():
    em = Emitter()
    em("// rho = sum f, j = sum f xi, e2f = sum f |xi|^2 (Sec. 3, macroscopic step).")
    em("template <class T, class A>")
    em("__device__ __forceinline__ void f_moments(const A& f, T& rho, T& jx, T& jy, T& jz,")
    em("                                          T& e2f) {")
    # pair sums / differences
    for i in range(1, Q, 2):
        em(f"  const T ps{i} = f[{i}] + f[{i + 1}], pd{i} = f[{i}] - f[{i + 1}];")
    em(f"  rho = f[0] + {tree_sum([f'ps{i}' for i in range(1, Q, 2)])};")
    for a, nm in enumerate(("jx", "jy", "jz")):
        terms = [((CX, CY, CZ)[a][i], f"pd{i}") for i in range(1, Q, 2)]
        em(f"  {nm} = {lincomb(terms, 'T')};")
    by_c2 = defaultdict(list)
    for i in range(1, Q, 2):
        by_c2[sum(c * c for c in VEL[i])].append(f"ps{i}")
    parts = []
    for c2, lst in sorted(by_c2.items()):
        em(f"  const T sh{c2} = {tree_sum(lst)};")
        parts.append((c2, f"sh{c2}"))
    em(f"  e2f = {lincomb(parts, 'T')};")
    em("}")
    em("")
    em("// sum g (the second population's share of the total energy).")
    em("template <class T, class A>")
    em("__device__ __forceinline__ T g_sum(const A& g) {")
    em(f"  const T gs = {tree_sum([f'g[{i}]' for i in range(Q)])};")
    em("  return gs;")
    em("}")
    return em.lines


def exp_constants():
    ln2 = D(2).ln()
    L = ln2 / 256
    inv = 256 / ln2
    # head with 32 significant bits so k*L_hi is exact for |k| < 2^21
    import math
    e = math.floor(math.log2(float(L)))
    scale = D(2) ** (31 - e)
    L_hi = (L * scale).to_integral_value(rounding=decimal.ROUND_HALF_EVEN) / scale
    L_lo = L - L_hi
    table = [D(2) ** (D(j) / 256) for j in range(256)]
    return float(inv), float(L_hi), float(L_lo), [float(t) for t in table]


def selfcheck(lines):
    """Evaluate the emitted straight-line code in Python on random inputs and compare with
    the direct sums over the 39 velocities."""
    import random
    import re
    rnd = random.Random(7)
    F = [rnd.uniform(0.1, 1.0) for _ in range(Q)]
    G = [rnd.uniform(0.1, 1.0) for _ in range(Q)]
    lam = [rnd.uniform(-1, 1) for _ in range(NM)]
    env = {"F": F, "f": F, "g": G, "l": lam, "fma": lambda a, b, c: a * b + c,
           "mul_rn": lambda a, b: a * b,
           "T": float, "double": float, "s": [0.0] * NM, "J": [0.0] * 91, "e": [0.0] * Q}
    for ln in lines:
        t = ln.strip()
        m = re.match(r"^(?:const\s+)?(?:T|double)\s+(.*);$", t)
        if m:
            for part in re.split(r",\s*(?=\w+\s*=)", m.group(1)):
                name, expr = part.split("=", 1)
                env[name.strip()] = eval(expr, env)
            continue
        m = re.match(r"^(\w+(?:\[\d+\])?)\s*(\+?=)\s*(.*);$", t)
        if m and not t.startswith(("//", "template", "__device__", "return")):
            tgt, op, expr = m.groups()
            val = eval(expr, env)
            mm = re.match(r"(\w+)\[(\d+)\]", tgt)
            if mm:
                arr, idx = mm.group(1), int(mm.group(2))
                env[arr][idx] = env[arr][idx] + val if op == "+=" else val
            else:
                env[tgt] = env[tgt] + val if op == "+=" else val
    for i in range(Q):
        ref = sum(lam[k] * phi(k, VEL[i]) for k in range(NM))
        assert abs(env["e"][i] - ref) < 1e-12, ("exponent", i)
    for k in range(NM):
        ref = sum(F[i] * phi(k, VEL[i]) for i in range(Q))
        assert abs(env["s"][k] - ref) < 1e-11, ("s", k, env["s"][k], ref)
        for l in range(k + 1):
            ref = sum(F[i] * phi(k, VEL[i]) * phi(l, VEL[i]) for i in range(Q))
            assert abs(env["J"][tri(k, l)] - ref) < 1e-9 * max(1, abs(ref)), ("J", k, l)
    rho = sum(F)
    assert abs(env["rho"] - rho) < 1e-12
    for a, nm in enumerate(("jx", "jy", "jz")):
        assert abs(env[nm] - sum(F[i] * VEL[i][a] for i in range(Q))) < 1e-12
    e2f = sum(F[i] * sum(c * c for c in VEL[i]) for i in range(Q))
    assert abs(env["e2f"] - e2f) < 1e-11
    assert abs(env["gs"] - sum(G)) < 1e-12


def strip_2d(lines):
    """The lines without the z-mirror functions (they reuse variable names)."""
    out, skip = [], False
    for ln in lines:
        if ln.startswith("__device__ __forceinline__ void exponents2d") or \
                ln.startswith("__device__ __forceinline__ void moments2d") or \
                ln.startswith("__device__ __forceinline__ void moments_s2d"):
            skip = True
        if not skip:
            out.append(ln)
        elif ln == "}":
            skip = False
    return out


def function_body(lines, start):
    out, on = [], False
    for ln in lines:
        if ln.startswith(start):
            on = True
            continue
        if on:
            if ln == "}":
                break
            out.append(ln)
    return out


def selfcheck_2d(lines):
    """The z-mirror functions on z-symmetric inputs against direct sums over the 39."""
    import random
    import re
    rnd = random.Random(11)
    mirror = {i: VEL.index((VEL[i][0], VEL[i][1], -VEL[i][2])) for i in range(Q)}
    F = [0.0] * Q
    for i in range(Q):
        if VEL[i][2] >= 0:
            F[i] = F[mirror[i]] = rnd.uniform(0.1, 1.0)
    lam = [rnd.uniform(-1, 1) if k in ZEVEN else 0.0 for k in range(NM)]
    env = {"F": F, "l": lam, "fma": lambda a, b, c: a * b + c, "mul_rn": lambda a, b: a * b,
           "T": float, "double": float,
           "s": [0.0] * N2, "J": [0.0] * (N2 * (N2 + 1) // 2), "e": [0.0] * Q}

    def run(body):
        for ln in body:
            t = ln.strip()
            m = re.match(r"^(?:const\s+)?(?:T|double)\s+(.*);$", t)
            if m:
                for part in re.split(r",\s*(?=\w+\s*=)", m.group(1)):
                    name, expr = part.split("=", 1)
                    env[name.strip()] = eval(expr, env)
                continue
            m = re.match(r"^(\w+)\[(\d+)\]\s*=\s*(.*);$", t)
            if m:
                env[m.group(1)][int(m.group(2))] = eval(m.group(3), env)
    run(function_body(lines, "__device__ __forceinline__ void exponents2d"))
    for i in range(Q):
        ref = sum(lam[k] * phi(k, VEL[i]) for k in range(NM))
        assert abs(env["e"][i] - ref) < 1e-12, ("exponent2d", i)
    run(function_body(lines, "__device__ __forceinline__ void moments2d"))
    for a, k in enumerate(ZEVEN):
        ref = sum(F[i] * phi(k, VEL[i]) for i in range(Q))
        assert abs(env["s"][a] - ref) < 1e-11, ("s2d", k)
        for b, l in enumerate(ZEVEN[:a + 1]):
            ref = sum(F[i] * phi(k, VEL[i]) * phi(l, VEL[i]) for i in range(Q))
            assert abs(env["J"][tri(a, b)] - ref) < 1e-9 * max(1, abs(ref)), ("J2d", k, l)
    env["s"] = [0.0] * N2
    run(function_body(lines, "__device__ __forceinline__ void moments_s2d"))
    for a, k in enumerate(ZEVEN):
        ref = sum(F[i] * phi(k, VEL[i]) for i in range(Q))
        assert abs(env["s"][a] - ref) < 1e-11, ("s_2d", k)
    # the z-odd sums vanish exactly on z-symmetric F (which the reduction relies on)
    for k in range(NM):
        if k not in ZEVEN:
            assert sum(F[i] * phi(k, VEL[i]) for i in range(Q)) == 0.0


def generate():
    """The lines of d3q39_gen.cuh, after the self-checks."""
    inv, L_hi, L_lo, table = exp_constants()
    lines = ["// d3q39_gen.cuh -- GENERATED by gen_d3q39.py; do not edit.",
             "#pragma once", "", "namespace lbm39 {", "namespace gen {", "",
             "// Rounded products that are never contracted into a fused multiply-add.",
             "__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }",
             "__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }",
             ""]
    lines += gen_exponents()
    lines.append("")
    exp2d = gen_exponents(zsym=True)
    lines += exp2d
    lines.append("")
    ml, nmono = gen_moments()
    lines += ml
    lines.append("")
    lines += gen_pop_moments()
    lines.append("")
    lines.append("// exp(x) = 2^(k/256) exp(r), x = k ln2/256 + r (table-driven method of P. T. P. Tang,")
    lines.append("// ACM TOMS 15(2), 1989, with a 256-entry table): 256/ln2, ln2/256 = head + tail.")
    lines.append(f"constexpr double EXP_INV_L = {inv!r};")
    lines.append(f"constexpr double EXP_L_HI = {L_hi!r};")
    lines.append(f"constexpr double EXP_L_LO = {L_lo!r};")
    lines.append("// 2^(j/256), j = 0..255, each the double nearest the exact value.")
    lines.append("__device__ __constant__ double kExp2Table[256] = {")
    for j in range(0, 256, 4):
        lines.append("    " + ", ".join(repr(t) for t in table[j:j + 4]) + ",")
    lines.append("};")
    lines += ["", "}  // namespace gen", "}  // namespace lbm39", ""]
    selfcheck(strip_2d(lines))
    selfcheck_2d(lines)
    return lines, nmono


def main():
    lines, nmono = generate()
    out = os.path.join(HERE, "d3q39_gen.cuh")
    with open(out, "w") as fh:
        fh.write("\n".join(lines))
    print(f"wrote {out}: {nmono} distinct monomials")


if __name__ == "__main__":
    main()
