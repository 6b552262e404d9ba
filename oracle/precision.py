"""Precision of the computation (oracle; test infrastructure only).

Sec. 2.5.  The paper delegates r_m to a lemma of another paper and N_m to an
algorithm of another paper, neither printed.  The readings used here:

* r_m (the relative precision of the columns of pole order m): the
  coefficients a_i of P(T), i <= b/2, satisfy |a_i| <= C(b, i) p^{(n-1)i/2}
  (Weil), so a_i is fixed by its residue mod p^{e_i}, e_i the least e with
  p^e > 2 C(b, i) p^{(n-1) i / 2}.  Write F = C diag(p^{sigma_j}) with
  sigma_j = n - m_j (Mazur's Newton over Hodge: C is integral).  If the
  columns of C of pole order m are known mod p^{r_m}, a principal minor of
  F on a column set I is known mod p^{sum_{j in I} sigma_j + min_{j in I}
  r_{m_j}}.  So it suffices that r_m >= e_i - G_m(i) for every i <= b/2,
  where G_m(i) = (n - m) + the sum of the i - 1 smallest slopes of the
  other columns: r_m = max(1, max_i (e_i - G_m(i))).  The paper states that
  r_m depends on m and p; this is the reading of how.
* N_m: the truncation error of Prop. 2.1 at N terms is a sum of integral
  forms of pole order p(m + i), i >= N, multiplied by p^{m-1+i}.  Reducing
  such a form to the basis costs at most LOSS(K) digits (a logarithmic bound
  in the pole order K).  N_m is the least N with m - 1 + i - LOSS(p(m+i)) >= r
  for all i >= N, with LOSS(K) = (n - 1) floor(log_p K).  For plane curves
  this is exactly the smallest N for which F mod p^r stops changing (checked
  at p = 7 and p = 11 for both pole orders); for n > 2 the factor n - 1 is
  a margin.  Pinned by point counts and by the stability of F under
  N_m -> N_m + 1.
* M = max_m (r + v_p((p s_m - 1)!) - m + 1), s_m = N_m + m - 1, as printed.
"""
from math import comb


def vp(x, p):
    if x == 0:
        raise ValueError("v_p(0)")
    e = 0
    while x % p == 0:
        x //= p
        e += 1
    return e


def vp_factorial(x, p):
    """Legendre: v_p(x!)."""
    e = 0
    t = p
    while t <= x:
        e += x // t
        t *= p
    return e


def hodge_polygon(n, pole_orders):
    """H(i) for i = 0..b: sums of the i smallest slopes n - m."""
    slopes = sorted(n - m for m in pole_orders)
    H = [0]
    for s in slopes:
        H.append(H[-1] + s)
    return H


def weil_digits(n, b, p, i):
    """Least e with p^e > 2 C(b, i) p^{(n-1) i / 2}; compared squared to stay in Z."""
    bound_sq = 4 * comb(b, i) ** 2 * p ** ((n - 1) * i)
    e = 0
    while p ** (2 * e) <= bound_sq:
        e += 1
    return e


def coefficient_digits(n, p, b):
    """[e_0, ..., e_{b//2}]: a_i is determined by a_i mod p^{e_i}."""
    return [weil_digits(n, b, p, i) for i in range(b // 2 + 1)]


def relative_precisions(n, p, pole_orders):
    """{m: r_m} for the pole orders present (see the module docstring)."""
    b = len(pole_orders)
    e = coefficient_digits(n, p, b)
    slopes = sorted(n - m for m in pole_orders)
    r = {}
    for m in sorted(set(pole_orders)):
        others = list(slopes)
        others.remove(n - m)
        best = 1
        for i in range(1, b // 2 + 1):
            G = (n - m) + sum(others[:i - 1])
            best = max(best, e[i] - G)
        r[m] = best
    return r


def ilog(K, p):
    """floor(log_p K) for K >= 1."""
    e = 0
    t = p
    while t <= K:
        t *= p
        e += 1
    return e


def loss(K, n, p):
    return (n - 1) * ilog(K, p)


def series_order(m, r, n, p):
    """Least N >= 1 with m - 1 + i - loss(p(m+i)) >= r for every i >= N.

    m - 1 + i - loss(p(m+i)) is nondecreasing in i except where the log
    jumps; checking up to the next power of p beyond the candidate covers
    every jump that can follow it.
    """
    N = 1
    while True:
        ok = True
        i = N
        limit = N + 4 * (n + 1) * (ilog(p * (m + N), p) + 2) + 8
        while i <= limit:
            if m - 1 + i - loss(p * (m + i), n, p) < r:
                ok = False
                break
            i += 1
        if ok:
            return N
        N += 1


class Precision:
    def __init__(self, n, d, p, pole_orders, r=None, N=None):
        """pole_orders: pole order m of each basis element.  r, N: optional overrides
        (an int for all m, or a dict m -> value) used by small parity cases."""
        self.n, self.d, self.p = n, d, p
        ms = sorted(set(pole_orders))
        self.e = coefficient_digits(n, p, len(pole_orders))
        if r is None:
            self.r = relative_precisions(n, p, pole_orders)
        elif isinstance(r, int):
            self.r = {m: r for m in ms}
        else:
            self.r = dict(r)
        if N is None:
            self.N = {m: series_order(m, self.r[m], n, p) for m in ms}
        elif isinstance(N, int):
            self.N = {m: N for m in ms}
        else:
            self.N = dict(N)
        self.s = {m: self.N[m] + m - 1 for m in ms}
        self.M = max(self.r[m] + vp_factorial(p * self.s[m] - 1, p) - m + 1 for m in ms)
        self.q = p ** self.M
