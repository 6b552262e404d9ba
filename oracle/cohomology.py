"""Griffiths-Dwork cohomology of U = P^n - V(f) (oracle; test infrastructure only).

Follows Sec. 2.2-2.3 (Griffiths-Dwork relations, monomial basis of the
cokernel of the Jacobian map M_k), Prop. 3.3 (the controlled-reduction map
R_{u,v}, for S = {0..n} and for a general S with f S-smooth, Definition 3.1)
and Sec. 3.3 step (2) (final reduction to the basis).

General S.  With J_S spanned by d_i f (i in S) and x_i d_i f (i not in S),
Prop. 3.3 writes x^v g / x^S = sum_{i in S} g_i d_i f + sum_{i not in S}
x_i g_i d_i f.  Put G_i = g_i for i in S and G_i = x_i g_i otherwise (a form
of degree kappa_S - d + 1, divisible by x_i when i is not in S); then both
sums of the printed R_{u,v} become x^S sum_i (u_i G_i / x_i + d_i G_i), and
a monomial x^nu of G_i with coefficient c contributes (u_i + nu_i) c to the
output monomial nu + 1_S - e_i.  kappa_S = deg(x^v g / x^S) = d + dn - n - |S|
= (n+1)(d-1) + 1 - |S|, the Macaulay degree of the n+1 generators of J_S
(|S| of degree d-1, the rest of degree d), so the section exists exactly
when f is S-smooth.  S = {0..n} is the smooth case of the same formulas.
"""
import numpy as np

from .algebra import (MonomialIndex, monomials, poly_deriv, poly_from_coeffs,
                      poly_mul, right_inverse_mod, pivot_columns_mod_p,
                      add_exp, sub_exp)


class Hypersurface:
    """f in Z[x_0..x_n]_d with coefficients in [0, p), lifted from F_p (Sec. 2.1)."""

    def __init__(self, n, d, p, coeffs):
        self.n, self.d, self.p = n, d, p
        self.nv = n + 1
        self.coeffs = list(coeffs)
        self.f = poly_from_coeffs(self.nv, d, coeffs)
        self.df = [poly_deriv(self.f, i) for i in range(self.nv)]

    def jacobian_matrix(self, k, S=None):
        """Matrix of M_k: (Homog_{k-d+1})^{n+1} -> Homog_k, (mu_i) -> sum mu_i d_i f.

        Rows: monomials of degree k; columns: pairs (i, nu) with i major and
        nu in monomial order (Sec. 2.3).  With S given, the map of J_S
        (Definition 3.1): for i not in S only the nu with nu_i >= 1 are
        columns (the multiples of x_i d_i f).
        """
        rows = MonomialIndex(self.nv, k)
        src = monomials(self.nv, k - self.d + 1)
        S = range(self.nv) if S is None else S
        cols = [(i, nu) for i in range(self.nv) for nu in src if i in S or nu[i] >= 1]
        M = [[0] * len(cols) for _ in range(len(rows))]
        for c, (i, nu) in enumerate(cols):
            for e, a in self.df[i].items():
                M[rows.pos[add_exp(e, nu)]][c] += a
        return M, rows, cols


def is_smooth(n, d, p, coeffs):
    """Jacobian criterion made linear: smooth iff M_k is onto for k = (n+1)(d-2)+1.

    Valid when p does not divide d: then f lies in the ideal of its
    partials (Euler), and the partials have no common projective zero iff
    they form a regular sequence, iff their ideal contains every form of
    degree (n+1)(d-2)+1 (Macaulay).
    """
    X = Hypersurface(n, d, p, coeffs)
    k = (n + 1) * (d - 2) + 1
    M, rows, _ = X.jacobian_matrix(k)
    return len(pivot_columns_mod_p(M, p)) == len(rows)


def full_S(n):
    return tuple(range(n + 1))


def kappa_S(n, d, S):
    """Degree of x^v g / x^S in Prop. 3.3: d + dn - n - |S| = (n+1)(d-1) + 1 - |S|."""
    return (n + 1) * (d - 1) + 1 - len(S)


def is_S_smooth(n, d, p, coeffs, S):
    """Definition 3.1: J_S defines the empty scheme, decided as for `is_smooth`.

    The n+1 generators of J_S have no common projective zero iff they form a
    regular sequence, iff their span contains every form of degree
    kappa_S (Macaulay: the sum of the degrees minus n).  S = {0..n} gives
    `is_smooth`.
    """
    X = Hypersurface(n, d, p, coeffs)
    k = kappa_S(n, d, S)
    M, rows, _ = X.jacobian_matrix(k, S)
    return len(pivot_columns_mod_p(M, p)) == len(rows)


def cohomology_basis(X):
    """Monomial basis B of H^n_dR(U) (Sec. 2.3).

    For m = 1..n and k = dm - n - 1, B_m = the monomials of degree k that are
    NOT pivot columns of the row echelon form (over F_p) of the matrix whose
    rows span the image of M_k, with columns in monomial order.  The pivot
    set depends only on that image and the column order, so the choice is
    canonical.  Returns a list of (m, beta) with m ascending, beta in
    monomial order.
    """
    basis = []
    for m in range(1, X.n + 1):
        k = X.d * m - X.n - 1
        mons = monomials(X.nv, k)
        if not mons:
            continue
        if k - X.d + 1 < 0:
            basis += [(m, b) for b in mons]
            continue
        M, rows, cols = X.jacobian_matrix(k)
        image_rows = [[M[r][c] for r in range(len(rows))] for c in range(len(cols))]
        piv = set(pivot_columns_mod_p(image_rows, X.p))
        basis += [(m, rows.mons[i]) for i in range(len(rows)) if i not in piv]
    return basis


def hodge_count(n, d):
    """dim H^n_dR(U) = ((d-1)^{n+1} + (-1)^{n+1}(d-1)) / d."""
    return ((d - 1) ** (n + 1) + (-1) ** (n + 1) * (d - 1)) // d


class Section:
    """Right inverse of the map of J_S in degree kappa_S over Z/q (Prop. 3.3 proof).

    For a monomial x^gamma of degree kappa_S, `solve(gamma)` returns
    G_0..G_n with sum G_i d_i f = x^gamma mod q, G_i divisible by x_i for i
    not in S (G_i = x_i g_i in the printed notation).  For S = {0..n},
    kappa = (n+1)(d-2)+1 and G_i = g_i in Homog_{n(d-2)}.  The decomposition is
    not unique; this one is Gauss-Jordan with unit pivots, columns (i, nu)
    visited in order, free variables zero.  `column_order` lets a test pick a
    different convention to check that results do not depend on it.
    """

    def __init__(self, X, q, column_order=None, S=None):
        self.X = X
        self.q = q
        self.S = full_S(X.n) if S is None else tuple(sorted(S))
        k = kappa_S(X.n, X.d, self.S)
        M, rows, cols = X.jacobian_matrix(k, self.S)
        if column_order is not None:
            M = [[row[c] for c in column_order] for row in M]
            cols = [cols[c] for c in column_order]
        Xinv, _ = right_inverse_mod(M, q, X.p)
        self.rows = rows
        self.cols = cols
        self.Xinv = Xinv
        self.cache = {}

    def solve(self, gamma):
        if gamma in self.cache:
            return self.cache[gamma]
        j = self.rows.pos[gamma]
        g = [dict() for _ in range(self.X.nv)]
        col = self.Xinv[:, j]
        for c, (i, nu) in enumerate(self.cols):
            a = int(col[c]) % self.q
            if a:
                g[i][nu] = a
        self.cache[gamma] = g
        return g


def R_matrix(X, sec, Sidx, u, v):
    """Matrix of R_{u,v} on Homog_{dn-n} (Prop. 3.3), mod q, for the section's S.

    For an input monomial x^mu: x^v x^mu / x^S = sum_i G_i d_i f via the
    section, and R_{u,v}(x^mu) = x^S sum_i (u_i G_i / x_i + d_i G_i): the
    monomial x^nu of G_i with coefficient a adds (u_i + nu_i) a at
    nu + 1_S - e_i.  Inputs with x^v x^mu / x^S not a polynomial have no
    image; they never carry a nonzero coefficient on a valid reduction path
    (their column is left zero and the driver asserts the coefficient is zero).
    """
    q = sec.q
    s = len(Sidx)
    R = np.zeros((s, s), dtype=object)
    oneS = tuple(1 if i in sec.S else 0 for i in range(X.nv))
    for c, mu in enumerate(Sidx.mons):
        gamma = sub_exp(add_exp(v, mu), oneS)
        if min(gamma) < 0:
            continue
        G = sec.solve(gamma)
        for i in range(X.nv):
            for nu, a in G[i].items():
                out = tuple(nu[t] + oneS[t] - (1 if t == i else 0) for t in range(X.nv))
                R[Sidx.pos[out], c] = (R[Sidx.pos[out], c] + (u[i] + nu[i]) * a) % q
    return R


def affine_parts(X, sec, Sidx, v):
    """A_0..A_{n+1} with R_{u,v} = sum_i A_i u_i + A_{n+1} (Sec. 3.1).

    R_{u,v} is affine in u by its definition (R_matrix): the monomial x^nu of
    G_i with coefficient a puts a into A_i and nu_i a into A_{n+1}, both at
    row nu + 1_S - e_i.
    """
    q = sec.q
    s = len(Sidx)
    parts = [np.zeros((s, s), dtype=object) for _ in range(X.nv + 1)]
    A_last = parts[X.nv]
    oneS = tuple(1 if i in sec.S else 0 for i in range(X.nv))
    for c, mu in enumerate(Sidx.mons):
        gamma = sub_exp(add_exp(v, mu), oneS)
        if min(gamma) < 0:
            continue
        G = sec.solve(gamma)
        for i in range(X.nv):
            Ai = parts[i]
            for nu, a in G[i].items():
                row = Sidx.pos[tuple(nu[t] + oneS[t] - (1 if t == i else 0) for t in range(X.nv))]
                Ai[row, c] = (Ai[row, c] + a) % q
                if nu[i]:
                    A_last[row, c] = (A_last[row, c] + nu[i] * a) % q
    return parts


class FinalReduction:
    """Sec. 3.3 step (2): reduce a pole-order-n numerator to the basis B.

    At pole order m' with numerator h in Homog_{dm'-n-1}: write
    h = sum_{beta in B_m'} c_beta x^beta + sum_i h_i d_i f; record c_beta;
    then h <- (1/(m'-1)) sum_i d_i h_i (Griffiths-Dwork) at pole order m'-1.
    The coefficients c_beta are unique; the h_i are not, but the class of
    sum_i d_i h_i is.
    """

    def __init__(self, X, basis, q):
        self.X, self.q = X, q
        self.basis = basis
        self.levels = {}
        for m in range(1, X.n + 1):
            k = X.d * m - X.n - 1
            rows = MonomialIndex(X.nv, k)
            if len(rows) == 0:
                continue
            Bm = [b for (mm, b) in basis if mm == m]
            cols = [('b', b) for b in Bm]
            M = [[0] * len(Bm) for _ in range(len(rows))]
            for c, b in enumerate(Bm):
                M[rows.pos[b]][c] = 1
            if k - X.d + 1 >= 0:
                J, _, jcols = X.jacobian_matrix(k)
                for r in range(len(rows)):
                    M[r] += J[r]
                cols += [('j', ij) for ij in jcols]
            Xinv, _ = right_inverse_mod(M, q, X.p)
            self.levels[m] = (rows, cols, Xinv)
        self.bpos = {mb: i for i, mb in enumerate(basis)}

    def reduce(self, h):
        """h: dict over Homog_{dn-n-1} (pole order n).  Returns coefficients on B."""
        X, q = self.X, self.q
        out = [0] * len(self.basis)
        for m in range(X.n, 0, -1):
            if m not in self.levels:
                continue
            rows, cols, Xinv = self.levels[m]
            vec = np.zeros(len(rows), dtype=object)
            for e, a in h.items():
                vec[rows.pos[e]] = a % q
            sol = Xinv.dot(vec) % q
            hi = [dict() for _ in range(X.nv)]
            for c, (kind, key) in enumerate(cols):
                a = int(sol[c])
                if not a:
                    continue
                if kind == 'b':
                    out[self.bpos[(m, key)]] = a
                else:
                    i, nu = key
                    hi[i][nu] = a
            if m == 1:
                break
            inv = pow(m - 1, -1, q)
            nh = {}
            for i in range(X.nv):
                for e, a in poly_deriv(hi[i], i).items():
                    nh[e] = (nh.get(e, 0) + a * inv) % q
            h = {e: a for e, a in nh.items() if a}
        return out
