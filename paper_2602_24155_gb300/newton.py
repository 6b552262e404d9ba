"""Newton polygons of zeta functions and a search for Newton strata over the batch engine.

The search follows the paper's Method 1 (Sec. 5.1, "fully random guessing"): draw random smooth hypersurfaces,
compute their zeta functions and keep those whose Newton polygon lies in the wanted stratum; since Newton strata
jump in codimension one, a stratum one step above the generic one is hit with probability about 1/p.  Before the
full computation a cheap filter discards ordinary instances: the same engine run at relative precision r = 1 gives
P(T) mod p, whose degree is the number of unit roots of Frobenius (the p-rank of the Jacobian for a curve, Sec. 2.5
and the Hodge polygon argument: only the columns of pole order n survive mod p).  Only instances with p-rank at
most `max_p_rank` go through the full-precision run.

Everything here is host-side bookkeeping around `zeta_batch`; the reduction runs in the library's kernels.
"""
from fractions import Fraction

import numpy as np

from . import zeta_batch


def vp(x, p):
    """p-adic valuation of a nonzero integer."""
    x = abs(int(x))
    v = 0
    while x % p == 0:
        x //= p
        v += 1
    return v


def newton_slopes(P, p):
    """Slopes (ascending, with multiplicity, as Fractions) of the Newton polygon of P(T) = sum a_i T^i, a_0 = 1:
    the lower convex hull of the points (i, v_p(a_i)) for a_i != 0.  The reciprocal roots of P have these
    p-adic valuations."""
    pts = [(i, vp(a, p)) for i, a in enumerate(P) if a != 0]
    if pts[0][0] != 0:
        raise ValueError("P(0) must be nonzero")
    hull = [pts[0]]
    for pt in pts[1:]:
        while len(hull) >= 2:
            (x1, y1), (x2, y2) = hull[-2], hull[-1]
            # drop the middle point if it lies on or above the segment hull[-2] -> pt
            if (y2 - y1) * (pt[0] - x1) >= (pt[1] - y1) * (x2 - x1):
                hull.pop()
            else:
                break
        hull.append(pt)
    slopes = []
    for (x1, y1), (x2, y2) in zip(hull, hull[1:]):
        slopes += [Fraction(y2 - y1, x2 - x1)] * (x2 - x1)
    return slopes


def polygon_label(slopes):
    """Compact label of a Newton polygon, e.g. '0^4 1/2^4 1^4'."""
    parts = []
    i = 0
    while i < len(slopes):
        j = i
        while j < len(slopes) and slopes[j] == slopes[i]:
            j += 1
        parts.append("%s^%d" % (slopes[i], j - i))
        i = j
    return " ".join(parts)


def unit_roots_mod_p(P_low, p):
    """Number of reciprocal roots of valuation 0 from P(T) mod p: the degree of P mod p."""
    deg = 0
    for i, a in enumerate(P_low):
        if int(a) % p:
            deg = i
    return deg


def hodge_numbers(n, d):
    """b_m for m = 1..n: the dimension of the Jacobian ring in degree dm - n - 1, the coefficient of that degree in
    (1 + t + ... + t^(d-2))^(n+1) (Sec. 2.3); the basis elements of pole order m have Hodge slope n - m."""
    poly = [1]
    for _ in range(n + 1):
        new = [0] * (len(poly) + d - 2)
        for i, a in enumerate(poly):
            for j in range(d - 1):
                new[i + j] += a
        poly = new
    return {m: (poly[d * m - n - 1] if 0 <= d * m - n - 1 < len(poly) else 0) for m in range(1, n + 1)}


def first_slope(n, d):
    """(h0, length): the first slope of the Hodge polygon, n - (largest pole order with a basis element), and the
    number of basis elements with that slope."""
    b = hodge_numbers(n, d)
    m_top = max(m for m, k in b.items() if k)
    return n - m_top, b[m_top]


def first_slope_length(P_low, p, h0, r=1):
    """How many reciprocal roots have p-adic valuation h0, the first Hodge slope, from P(T) computed at relative
    precision r (a_i known mod p^(r + H(i)), H the Hodge polygon).  The Newton polygon lies on or above the Hodge
    polygon, whose first segment has slope h0, so that number is the largest i with v_p(a_i) = h0 i, and
    a_i mod p^(r + h0 i) decides it.  h0 = 0 (curves, K3 surfaces): the p-rank, the degree of P mod p.  h0 = 1
    (cubic threefolds, Hodge numbers 0, 5, 5, 0): the length of the slope-one segment, the p-rank of the
    intermediate Jacobian (Sec. 1.2); 5 is ordinary, 4 almost ordinary."""
    best = 0
    for i in range(1, len(P_low)):
        a = int(P_low[i]) % p ** (r + h0 * i)
        if a and vp(a, p) == h0 * i:
            best = i
    return best


def random_hypersurfaces(n, d, p, count, seed):
    """`count` random dense coefficient vectors (C(n+d, n) values in [0, p)) from numpy's PCG64 with `seed`."""
    from math import comb
    rng = np.random.Generator(np.random.PCG64(seed))
    m = comb(n + d, n)
    return [(n, d, p, [int(v) for v in rng.integers(0, p, m)]) for _ in range(count)]


def search(ctx, n, d, p, count, seed=0, max_p_rank=None, policy="p_chunk", path="vector"):
    """Method 1: random smooth hypersurfaces of degree d in P^n over F_p.

    Returns a dict: 'drawn', 'smooth', 'p_rank' (histogram over the smooth ones, from the r = 1 run, of the number
    of roots on the first Hodge slope: the p-rank for curves, the slope-one length for cubic threefolds), 'kept'
    (the instances with that number <= max_p_rank, default: one below the ordinary value, i.e. the non-ordinary
    ones), and 'strata' (Newton polygon label -> list of (coefficients, P) of the kept instances, from the
    full-precision run)."""
    specs = random_hypersurfaces(n, d, p, count, seed)
    low, per, _ = zeta_batch(ctx, specs, policy=policy, path=path, r=1)
    smooth = [i for i, x in enumerate(per) if x["status"] == 0]
    h0, ordinary = first_slope(n, d)
    ranks = {i: first_slope_length(low[i], p, h0) for i in smooth}
    if max_p_rank is None:
        max_p_rank = ordinary - 1
    kept = [i for i in smooth if ranks[i] <= max_p_rank]
    strata = {}
    if kept:
        full, per_full, _ = zeta_batch(ctx, [specs[i] for i in kept], policy=policy, path=path)
        for i, P in zip(kept, full):
            lab = polygon_label(newton_slopes(P, p))
            strata.setdefault(lab, []).append((specs[i][3], P))
    hist = {}
    for i in smooth:
        hist[ranks[i]] = hist.get(ranks[i], 0) + 1
    return {"drawn": count, "smooth": len(smooth), "p_rank": dict(sorted(hist.items())), "kept": len(kept),
            "strata": strata}


def k3_height(P, p, r=1):
    """Height of a K3 surface (b = 21) from P(T) computed at relative precision r.

    The Hodge polygon of a K3 has height H(i) = i - 1 at 1 <= i <= 20, so a_i is known mod p^(r + i - 1).  A K3 of
    finite height h has Newton slopes 1 - 1/h (h times), 1, 1 + 1/h (h times): its polygon passes through (h, h - 1)
    and lies strictly above the line y = i - 1 before it, so h is the least i with v_p(a_i) <= i - 1, which a_i mod p^i
    decides.  Returns h in 1..10, or None when no i <= 10 qualifies (supersingular: h is 1..10 or infinite)."""
    for i in range(1, 11):
        a = int(P[i]) % p ** (r + i - 1)
        if a and vp(a, p) <= i - 1:
            return i
    return None


def hodge_polygon(n, d):
    """H(i), i = 0..b: the Hodge polygon's height, the sum of the i smallest Hodge slopes (n - m for the basis
    elements of pole order m)."""
    slopes = []
    for m, k in sorted(hodge_numbers(n, d).items(), reverse=True):
        slopes += [n - m] * k
    H = [0]
    for sl in slopes:
        H.append(H[-1] + sl)
    return H


def fourfold_height(P, p, r=1):
    """Height of a cubic fourfold (Hodge numbers 1, 20, 1 on primitive H^4: a K3 surface's shape with every slope
    raised by one) from P(T) at relative precision r.  The Hodge polygon has H(i) = 2i - 1 for 1 <= i <= 21, so a_i
    is known mod p^(r + 2i - 1).  A fourfold of finite height h has Newton slopes 2 - 1/h (h times), 2, ..., 2 + 1/h
    (h times): its polygon passes through (h, 2h - 1) and lies strictly above y = 2i - 1 before it, so h is the
    least i with v_p(a_i) <= 2i - 1, which a_i mod p^(2i) decides.  Returns h in 1..11, or None (supersingular)."""
    for i in range(1, 12):
        a = int(P[i]) % p ** (r + 2 * i - 1)
        if a and vp(a, p) <= 2 * i - 1:
            return i
    return None


def k3_heights(ctx, specs, policy="p_chunk", path="vector"):
    """Heights of quartic K3 surfaces from one precision-1 batch.  Returns (heights, per-instance stats, total stats):
    heights[i] is 1..10, 'inf' for a supersingular surface, or None if the instance failed (e.g. not smooth)."""
    P_low, per, tot = zeta_batch(ctx, specs, policy=policy, path=path, r=1)
    out = []
    for spec, P in zip(specs, P_low):
        if P is None:
            out.append(None)
        else:
            h = k3_height(P, spec[2])
            out.append("inf" if h is None else h)
    return out, per, tot
