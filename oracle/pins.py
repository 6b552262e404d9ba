"""Independent checks that pin the oracle (test infrastructure only).

None of these use the controlled-reduction machinery:
  * point counts #X(F_{p^r}) by evaluating f on every point of P^n(F_{p^r})
    (own table arithmetic for F_{p^r});
  * Weil's Gauss-sum formula for diagonal hypersurfaces x_0^d + ... + x_n^d
    over F_p with p = 1 mod d (Ireland-Rosen ch. 8);
  * the Hasse-Witt matrix from f^{p-1}, which gives P(T) mod p;
  * Weil's bounds and the zeta function's relation to point counts
    (Sec. 1.1 and Sec. 2.1: Z = P^{(-1)^n} / prod_{i<n}(1 - p^i T)).
"""
from itertools import product
from math import comb

import numpy as np

from .algebra import monomials, poly_from_coeffs, poly_powers


# ---------------------------------------------------------------------------
# F_{p^r} by tables
# ---------------------------------------------------------------------------
def _prime_factors(x):
    out, t = [], 2
    while t * t <= x:
        if x % t == 0:
            out.append(t)
            while x % t == 0:
                x //= t
        t += 1
    if x > 1:
        out.append(x)
    return out


def _polmulmod(a, b, mod_poly, p):
    """Product of coefficient lists (low degree first) modulo a monic polynomial."""
    r = len(mod_poly) - 1
    res = [0] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        if x:
            for j, y in enumerate(b):
                res[i + j] = (res[i + j] + x * y) % p
    for k in range(len(res) - 1, r - 1, -1):
        c = res[k]
        if c:
            for t in range(r + 1):
                res[k - r + t] = (res[k - r + t] - c * mod_poly[t]) % p
    res = res[:r] + [0] * max(0, r - len(res))
    return res[:r]


class GF:
    """F_q, q = p^r; elements are integers sum c_i p^i (c_i = coefficient of x^i)."""

    def __init__(self, p, r):
        self.p, self.r, self.q = p, r, p ** r
        q = self.q
        self.poly = self._primitive_poly()
        # exp / log tables of the primitive element x
        exp = np.zeros(q - 1, dtype=np.int64)
        cur = [1] + [0] * (r - 1)
        xpoly = [0, 1] if r > 1 else None
        for k in range(q - 1):
            exp[k] = sum(c * p ** i for i, c in enumerate(cur))
            if r == 1:
                cur = [(cur[0] * self.gen1) % p]
            else:
                cur = _polmulmod(cur, xpoly, self.poly, p)
        self.exp = exp
        log = np.full(q, -1, dtype=np.int64)
        log[exp] = np.arange(q - 1)
        assert (log[1:] >= 0).all()
        self.log = log
        digits = np.zeros((q, r), dtype=np.int64)
        t = np.arange(q)
        for i in range(r):
            digits[:, i] = t % p
            t = t // p
        self.digits = digits
        self.weights = p ** np.arange(r)

    def _primitive_poly(self):
        p, r, q = self.p, self.r, self.p ** self.r
        if r == 1:
            for g in range(2, p):
                if all(pow(g, (p - 1) // l, p) != 1 for l in _prime_factors(p - 1)):
                    self.gen1 = g
                    return [0, 1]
            self.gen1 = 1
            return [0, 1]
        for tail in product(range(p), repeat=r):
            poly = list(tail) + [1]
            if poly[0] == 0:
                continue

            def xpow(e):
                res, base = [1] + [0] * (r - 1), [0, 1] + [0] * (r - 2)
                while e:
                    if e & 1:
                        res = _polmulmod(res, base, poly, p)
                    base = _polmulmod(base, base, poly, p)
                    e >>= 1
                return res

            one = [1] + [0] * (r - 1)
            if xpow(q - 1) != one:
                continue
            if all(xpow((q - 1) // l) != one for l in _prime_factors(q - 1)):
                return poly
        raise RuntimeError("no primitive polynomial")

    def mul(self, a, b):
        a = np.asarray(a)
        b = np.asarray(b)
        z = (a == 0) | (b == 0)
        la = self.log[np.where(z, 1, a)]
        lb = self.log[np.where(z, 1, b)]
        return np.where(z, 0, self.exp[(la + lb) % (self.q - 1)])

    def add(self, a, b):
        da = self.digits[np.asarray(a)]
        db = self.digits[np.asarray(b)]
        return ((da + db) % self.p) @ self.weights

    def powk(self, a, k):
        a = np.asarray(a)
        if k == 0:
            return np.ones_like(a)
        z = a == 0
        la = self.log[np.where(z, 1, a)]
        return np.where(z, 0, self.exp[(la * k) % (self.q - 1)])

    def elements(self):
        return np.arange(self.q)


def count_points(n, d, p, coeffs, r, chunk=1 << 20):
    """#X(F_{p^r}) for X = V(f) in P^n by evaluating f on every point."""
    K = GF(p, r)
    q = K.q
    mons = monomials(n + 1, d)
    terms = [(m, c) for m, c in zip(mons, coeffs) if c % p]
    total = 0
    # representatives: first nonzero coordinate equal to 1, at position lead
    for lead in range(n + 1):
        free = n - lead           # coordinates after the leading 1
        npts = q ** free
        for start in range(0, npts, chunk):
            idx = np.arange(start, min(npts, start + chunk), dtype=np.int64)
            coords = []
            for i in range(n + 1):
                if i < lead:
                    coords.append(np.zeros_like(idx))
                elif i == lead:
                    coords.append(np.ones_like(idx))
                else:
                    pos = n - i
                    coords.append((idx // q ** pos) % q)
            val = np.zeros_like(idx)
            for m, c in terms:
                t = np.full_like(idx, c % p)
                for i in range(n + 1):
                    if m[i]:
                        t = K.mul(t, K.powk(coords[i], m[i]))
                val = K.add(val, t)
            total += int((val == 0).sum())
    return total


def counts_to_charpoly_prefix(n, p, counts):
    """First len(counts) coefficients a_1.. of P(T) from #X(F_{p^r}), r = 1..R.

    #X(F_{p^r}) = sum_{i<n} p^{ir} + (-1)^{n+1} sum_j alpha_j^r and
    P(T) = prod (1 - alpha_j T); Newton's identities give a_1..a_R.
    """
    R = len(counts)
    s = []
    for r_, N in enumerate(counts, start=1):
        base = sum(p ** (i * r_) for i in range(n))
        s.append(((N - base) * (-1) ** (n + 1)))
    a = [1]
    for k in range(1, R + 1):
        # k a_k = -sum_{i=1}^{k} s_i a_{k-i}
        tot = sum(s[i - 1] * a[k - i] for i in range(1, k + 1))
        assert tot % k == 0
        a.append(-tot // k)
    return a


def charpoly_to_counts(n, p, P, R):
    """#X(F_{p^r}) for r = 1..R predicted by P(T) (inverse of the above)."""
    b = len(P) - 1
    s = []
    for k in range(1, R + 1):
        # s_k = -k a_k - sum_{i=1}^{k-1} s_i a_{k-i}
        ak = P[k] if k <= b else 0
        tot = -k * ak - sum(s[i - 1] * (P[k - i] if k - i <= b else 0) for i in range(1, k))
        s.append(tot)
    return [sum(p ** (i * r) for i in range(n)) + (-1) ** (n + 1) * s[r - 1]
            for r in range(1, R + 1)]


# ---------------------------------------------------------------------------
# Diagonal hypersurfaces: Gauss sums over F_p, p = 1 mod d
# ---------------------------------------------------------------------------
def fermat_charpoly(n, d, p, dps=80):
    """P(T) of x_0^d + ... + x_n^d over F_p for p = 1 mod d.

    Counting solutions with additive characters gives
    #X(F_p) = sum_{i<n} p^i + (1/p) sum_a prod_i g(chi^{a_i}),
    a in {1..d-1}^{n+1} with sum a_i = 0 mod d, chi of order d, g the
    Gauss sum.  Hasse-Davenport lifts this to every F_{p^r}, so the
    reciprocal roots of P are alpha(a) = (-1)^{n+1} p^{-1} prod_i g(chi^{a_i}).
    """
    import mpmath
    assert (p - 1) % d == 0
    mpmath.mp.dps = dps
    g0 = None
    for g in range(2, p):
        if all(pow(g, (p - 1) // l, p) != 1 for l in _prime_factors(p - 1)):
            g0 = g
            break
    ind = {}
    x = 1
    for k in range(p - 1):
        ind[x] = k
        x = (x * g0) % p
    zp = [mpmath.expjpi(mpmath.mpf(2 * t) / p) for t in range(p)]

    def gauss(a):
        return mpmath.fsum(mpmath.expjpi(mpmath.mpf(2 * a * ind[t]) / d) * zp[t]
                           for t in range(1, p))

    G = {a: gauss(a) for a in range(1, d)}
    roots = []
    for a in product(range(1, d), repeat=n + 1):
        if sum(a) % d:
            continue
        val = mpmath.mpf(1)
        for ai in a:
            val *= G[ai]
        roots.append((-1) ** (n + 1) * val / p)
    poly = [mpmath.mpc(1)]
    for al in roots:
        new = poly + [mpmath.mpc(0)]
        for i in range(len(poly)):
            new[i + 1] -= al * poly[i]
        poly = new
    out = []
    for c in poly:
        re = int(mpmath.nint(c.real))
        assert abs(c.real - re) < mpmath.mpf(10) ** (-dps // 3)
        assert abs(c.imag) < mpmath.mpf(10) ** (-dps // 3)
        out.append(re)
    return out


# ---------------------------------------------------------------------------
# Hasse-Witt matrix: P(T) mod p
# ---------------------------------------------------------------------------
def hasse_witt_charpoly_mod_p(n, d, p, coeffs):
    """det(1 - T H) mod p for the Hasse-Witt matrix H of X = V(f).

    H^{n-1}(X, O_X) has the basis of monomials x^beta with all beta_i >= 1
    and |beta| = d; Frobenius acts by H[beta, beta'] = coefficient of
    x^{p beta' - beta} in f^{p-1}.  Only the slope-0 part of Frobenius
    survives mod p, so P(T) = det(1 - T H) mod p.
    """
    f = poly_from_coeffs(n + 1, d, coeffs)
    fp1 = poly_powers({e: c % p for e, c in f.items()}, p - 1)[p - 1]
    interior = [m for m in monomials(n + 1, d) if min(m) >= 1]
    h = len(interior)
    H = [[0] * h for _ in range(h)]
    for i, bi in enumerate(interior):
        for j, bj in enumerate(interior):
            e = tuple(p * y - x for x, y in zip(bi, bj))
            H[i][j] = fp1.get(e, 0) % p
    # det(1 - T H) mod p via det(T I - H) reversed (Berkowitz over Z, then mod p)
    from .algebra import berkowitz_charpoly
    cp = berkowitz_charpoly(H)
    return [c % p for c in cp]


# ---------------------------------------------------------------------------
# Weil checks on P(T)
# ---------------------------------------------------------------------------
def _squarefree_part(P):
    """P / gcd(P, P') for an integer polynomial (list, constant term first), exact over Q."""
    from fractions import Fraction

    def trim(a):
        while len(a) > 1 and a[-1] == 0:
            a = a[:-1]
        return a

    def divmod_poly(a, b):
        a = [Fraction(x) for x in a]
        q = [Fraction(0)] * max(1, len(a) - len(b) + 1)
        while len(a) >= len(b) and any(a):
            c = a[-1] / b[-1]
            k = len(a) - len(b)
            q[k] = c
            for i, bi in enumerate(b):
                a[i + k] -= c * bi
            a = trim(a[:-1]) if len(a) > 1 else a
        return trim(q), trim(a)

    A = trim([Fraction(x) for x in P])
    D = trim([i * A[i] for i in range(1, len(A))]) or [Fraction(0)]
    g, h = A, D
    while any(h):
        _, r = divmod_poly(g, h)
        g, h = h, r
    g = [x / g[-1] for x in g]
    q, r = divmod_poly(A, g)
    assert not any(r)
    return q


def root_moduli_ok(n, p, P, tol=1e-20, dps=60):
    """Every reciprocal root of P has absolute value p^{(n-1)/2}.

    Repeated roots (p zeta with zeta a root of unity occurs several times on
    special surfaces) are removed first: the roots of the square-free part
    P / gcd(P, P') are the distinct roots of P."""
    import mpmath
    mpmath.mp.dps = dps
    Q = _squarefree_part(P)
    # reciprocal roots alpha of P are the roots of T^b P(1/T) = sum a_i T^{b-i}
    coeffs = [mpmath.mpf(x.numerator) / x.denominator for x in Q]
    if len(coeffs) == 1:
        return True
    roots = mpmath.polyroots(coeffs, maxsteps=400, extraprec=400)
    target = mpmath.mpf(p) ** (mpmath.mpf(n - 1) / 2)
    return all(abs(abs(r) / target - 1) < mpmath.mpf(10) ** -12 for r in roots) and len(roots) == len(Q) - 1


def newton_above_hodge(n, p, P, pole_orders):
    """v_p(a_i) >= H(i) for all i, with equality at i = b (Mazur)."""
    from .precision import hodge_polygon, vp
    H = hodge_polygon(n, pole_orders)
    b = len(P) - 1
    for i in range(1, b + 1):
        if P[i] != 0 and vp(P[i], p) < H[i]:
            return False
    return vp(P[b], p) == H[b]
