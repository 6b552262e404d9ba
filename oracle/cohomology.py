"""Griffiths-Dwork cohomology of U = P^n - V(f) (oracle; test infrastructure only).

Follows Sec. 2.2-2.3 (Griffiths-Dwork relations, monomial basis of the
cokernel of the Jacobian map M_k), Prop. 3.3 (the controlled-reduction map
R_{u,v} for S = {0..n}) and Sec. 3.3 step (2) (final reduction to the basis).
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

    def jacobian_matrix(self, k):
        """Matrix of M_k: (Homog_{k-d+1})^{n+1} -> Homog_k, (mu_i) -> sum mu_i d_i f.

        Rows: monomials of degree k; columns: pairs (i, nu) with i major and
        nu in monomial order (Sec. 2.3).
        """
        rows = MonomialIndex(self.nv, k)
        src = monomials(self.nv, k - self.d + 1)
        cols = [(i, nu) for i in range(self.nv) for nu in src]
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
    """Right inverse of M_kappa over Z/q, kappa = (n+1)(d-2)+1 (Prop. 3.3 proof).

    For a monomial x^gamma of degree kappa, `solve(gamma)` returns g_0..g_n in
    Homog_{n(d-2)} with sum g_i d_i f = x^gamma mod q.  The decomposition is
    not unique; this one is Gauss-Jordan with unit pivots, columns (i, nu)
    visited in order, free variables zero.  `column_order` lets a test pick a
    different convention to check that results do not depend on it.
    """

    def __init__(self, X, q, column_order=None):
        self.X = X
        self.q = q
        k = X.nv * (X.d - 2) + 1
        M, rows, cols = X.jacobian_matrix(k)
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
    """Matrix of R_{u,v} on Homog_{dn-n} (Prop. 3.3 with S = {0..n}), mod q.

    For an input monomial x^mu: x^v x^mu / x^S = sum_i g_i d_i f via the
    section, and R_{u,v}(x^mu) = x^S sum_i (u_i g_i + x_i d_i g_i) / x_i.
    Inputs with v_i + mu_i = 0 for some i have no polynomial x^v x^mu / x^S;
    they never carry a nonzero coefficient on a valid reduction path (their
    column is left zero and the driver asserts the coefficient is zero).
    """
    q = sec.q
    s = len(Sidx)
    R = np.zeros((s, s), dtype=object)
    one = (1,) * X.nv
    for c, mu in enumerate(Sidx.mons):
        gamma = sub_exp(add_exp(v, mu), one)
        if min(gamma) < 0:
            continue
        g = sec.solve(gamma)
        for i in range(X.nv):
            # h_i = u_i g_i + x_i d_i g_i, then multiply by x^S / x_i
            h = {}
            for nu, a in g[i].items():
                h[nu] = h.get(nu, 0) + u[i] * a
            for nu, a in poly_deriv(g[i], i).items():
                nu2 = nu[:i] + (nu[i] + 1,) + nu[i + 1:]
                h[nu2] = h.get(nu2, 0) + a
            for nu, a in h.items():
                out = tuple(nu[t] + (0 if t == i else 1) for t in range(X.nv))
                R[Sidx.pos[out], c] = (R[Sidx.pos[out], c] + a) % q
    return R


def affine_parts(X, sec, Sidx, v):
    """A_0..A_{n+1} with R_{u,v} = sum_i A_i u_i + A_{n+1} (Sec. 3.1).

    R_{u,v} is affine in u by its definition, so A_{n+1} = R_{0,v} and
    A_i = R_{e_i,v} - R_{0,v}.
    """
    q = sec.q
    zero = (0,) * X.nv
    R0 = R_matrix(X, sec, Sidx, zero, v)
    parts = []
    for i in range(X.nv):
        ei = tuple(1 if t == i else 0 for t in range(X.nv))
        parts.append((R_matrix(X, sec, Sidx, ei, v) - R0) % q)
    parts.append(R0)
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
