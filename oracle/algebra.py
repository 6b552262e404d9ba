"""Monomials, polynomials and linear algebra over Z/p^k (oracle; test infrastructure only).

Monomial order everywhere: descending lexicographic order of the exponent
vector (x_0 first).  Polynomials are dicts {exponent tuple: integer}.
"""
import numpy as np


def monomials(nvars, deg):
    """All exponent vectors of total degree `deg` in `nvars` variables, descending lex.

    Homog_deg of Sec. 2.1; empty for deg < 0 (the paper's convention).
    """
    if deg < 0:
        return []
    if nvars == 1:
        return [(deg,)]
    out = []
    for e0 in range(deg, -1, -1):
        for rest in monomials(nvars - 1, deg - e0):
            out.append((e0,) + rest)
    return out


class MonomialIndex:
    """Position of each monomial of one degree in the descending-lex order."""

    def __init__(self, nvars, deg):
        self.nvars = nvars
        self.deg = deg
        self.mons = monomials(nvars, deg)
        self.pos = {m: i for i, m in enumerate(self.mons)}

    def __len__(self):
        return len(self.mons)


def add_exp(a, b):
    return tuple(x + y for x, y in zip(a, b))


def sub_exp(a, b):
    return tuple(x - y for x, y in zip(a, b))


def poly_from_coeffs(nvars, deg, coeffs):
    """Polynomial dict from a coefficient list in the module's monomial order."""
    return {m: c for m, c in zip(monomials(nvars, deg), coeffs) if c}


def poly_mul(a, b, mod=None):
    out = {}
    for ea, ca in a.items():
        for eb, cb in b.items():
            e = add_exp(ea, eb)
            out[e] = out.get(e, 0) + ca * cb
    if mod is not None:
        out = {e: c % mod for e, c in out.items() if c % mod}
    else:
        out = {e: c for e, c in out.items() if c}
    return out


def poly_add(a, b, mod=None):
    out = dict(a)
    for e, c in b.items():
        out[e] = out.get(e, 0) + c
    if mod is not None:
        return {e: c % mod for e, c in out.items() if c % mod}
    return {e: c for e, c in out.items() if c}


def poly_scale(a, s, mod=None):
    if mod is not None:
        return {e: (c * s) % mod for e, c in a.items() if (c * s) % mod}
    return {e: c * s for e, c in a.items() if c * s}


def poly_deriv(a, i):
    """Partial derivative d/dx_i."""
    out = {}
    for e, c in a.items():
        if e[i] > 0:
            e2 = e[:i] + (e[i] - 1,) + e[i + 1:]
            out[e2] = out.get(e2, 0) + c * e[i]
    return {e: c for e, c in out.items() if c}


def poly_times_monomial(a, mono):
    return {add_exp(e, mono): c for e, c in a.items()}


def poly_powers(f, jmax):
    """[f^0, f^1, ..., f^jmax] with exact integer coefficients."""
    nv = len(next(iter(f)))
    out = [{(0,) * nv: 1}]
    for _ in range(jmax):
        out.append(poly_mul(out[-1], f))
    return out


def inv_mod(a, q):
    return pow(a, -1, q)


def right_inverse_mod(M, q, p):
    """X with M X = I mod q for a matrix M (rows x cols) of full row rank mod p.

    Gauss-Jordan elimination over Z/q, q = p^k: columns are visited in order
    and the pivot is the first remaining row whose entry is a unit; free
    variables are set to zero.  Returns (X, pivot_columns) with X a
    cols x rows object array.  Raises ValueError if the rank mod p is short.
    When q^2 < 2^62 the same elimination runs in int64 (every product of two
    residues is exact there); otherwise in Python integers.
    """
    A = np.array(M, dtype=object) % q
    r, c = A.shape
    small = q * q < (1 << 62)
    dt = np.int64 if small else object
    if small:
        A = A.astype(np.int64)
    E = np.zeros((r, r), dtype=dt)
    for i in range(r):
        E[i, i] = 1
    aug = np.concatenate([A, E], axis=1)
    pivcols = []
    rank = 0
    for col in range(c):
        if rank == r:
            break
        piv = None
        for i in range(rank, r):
            if aug[i, col] % p:
                piv = i
                break
        if piv is None:
            continue
        if piv != rank:
            aug[[rank, piv]] = aug[[piv, rank]]
        aug[rank] = (aug[rank] * inv_mod(int(aug[rank, col]), q)) % q
        factors = aug[:, col].copy()
        factors[rank] = 0
        nz = [i for i in range(r) if factors[i] % q]
        if nz:
            aug[nz] = (aug[nz] - np.outer(factors[nz], aug[rank])) % q
        pivcols.append(col)
        rank += 1
    if rank < r:
        raise ValueError("matrix is not of full row rank mod p")
    X = np.zeros((c, r), dtype=object)
    for k, col in enumerate(pivcols):
        X[col, :] = [int(a) for a in aug[k, c:]]
    return X, pivcols


def pivot_columns_mod_p(M, p):
    """Pivot columns of the row echelon form of M over F_p (columns in order).

    The set of pivot columns depends only on the row space of M and the
    column order, not on the elimination used.
    """
    A = np.array(M, dtype=np.int64) % p
    if A.size == 0:
        return []
    r, c = A.shape
    pivcols = []
    rank = 0
    for col in range(c):
        if rank == r:
            break
        nz = np.nonzero(A[rank:, col])[0]
        if len(nz) == 0:
            continue
        piv = rank + int(nz[0])
        if piv != rank:
            A[[rank, piv]] = A[[piv, rank]]
        A[rank] = (A[rank] * pow(int(A[rank, col]), -1, p)) % p
        below = A[rank + 1:, col].copy()
        if below.any():
            A[rank + 1:] = (A[rank + 1:] - np.outer(below, A[rank])) % p
        pivcols.append(col)
        rank += 1
    return pivcols


def rank_mod_p(M, p):
    return len(pivot_columns_mod_p(M, p))


def matmul_mod(A, B, q):
    """Exact product of object (or int) matrices, reduced mod q."""
    return (np.array(A, dtype=object).dot(np.array(B, dtype=object))) % q


def berkowitz_charpoly(F):
    """Coefficients [c_0, ..., c_b] of det(T*I - F) over Z, division-free.

    Berkowitz's algorithm (Berkowitz 1984): only ring operations, so exact on
    integer matrices.  c_0 = 1 is the leading coefficient.
    """
    F = [[int(x) for x in row] for row in F]
    b = len(F)
    if b == 0:
        return [1]
    # Vector of the characteristic polynomial of the leading r x r block,
    # built for r = 1..b via Toeplitz products.
    poly = [1, -F[0][0]]
    for r in range(1, b):
        # Partition leading (r+1)x(r+1) block: [[A, R], [C, a]] with A r x r.
        a = F[r][r]
        R = [F[i][r] for i in range(r)]      # column above the diagonal
        C = [F[r][j] for j in range(r)]      # row left of the diagonal
        A = [row[:r] for row in F[:r]]
        # Toeplitz column: t_0 = 1, t_1 = -a, t_{k+2} = -C A^k R
        t = [1, -a]
        vec = R[:]
        for _ in range(r):
            t.append(-sum(C[j] * vec[j] for j in range(r)))
            vec = [sum(A[i][j] * vec[j] for j in range(r)) for i in range(r)]
        # new poly = T * poly (lower-triangular Toeplitz of size (r+2)x(r+1))
        new = []
        for i in range(r + 2):
            s = 0
            for j in range(max(0, i - (len(t) - 1)), min(i, r) + 1):
                s += t[i - j] * poly[j]
            new.append(s)
        poly = new
    return poly
