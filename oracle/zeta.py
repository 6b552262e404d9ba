"""Zeta function of a smooth hypersurface by controlled reduction (oracle; test infrastructure only).

The end-to-end computation of Sec. 2-4 on the CPU with exact integers:
  1. smoothness (Jacobian criterion), monomial basis B (Sec. 2.3)
  2. precision r, N_m, M (Sec. 2.5; readings in oracle.precision)
  3. Frobenius expansion (Prop. 2.1): terms x^gamma / (x^S f^{p(m+j)}),
     gamma = p(beta+alpha+1) - 1 + 1_S
  4. Tweak (Alg. 1) into (u, g), terms with equal u combined
  5. a reduction policy (Sec. 4) plays the game of Sec. 3.4; each chunk is
     evaluated with Algorithm 2 on R_{x+yv,v} = y A + B (Prop. 3.3, Sec. 3.2)
  6. final Griffiths-Dwork reduction to B (Sec. 3.3 step (2))
  7. normalisation to the matrix F of p^{-1} sigma, P(T) = det(1 - T F),
     lift to Z[T] with the functional equation (Sec. 2.1).

Denominators.  A step from pole order K+1 to K divides by K (Prop. 3.3:
m x^{u+v} g / f^{m+1} = x^u R(g) / f^m).  The oracle runs every step without
the division and instead multiplies the term of pole order p(m+j) by
(p s_m - 1)! / (p(m+j) - 1)!, so every term of a column ends with the common
denominator (p s_m - 1)! / (n-1)!.  The unnormalised column Y is therefore
exactly ((p s_m - 1)! / (n-1)!) p^{1-m} times the coordinates of the
truncated expansion; it does not depend on the policy or on the section,
only on B, N_m and M.  Dividing it out is exact, which is why the algorithm
precision is M = r + v_p((p s_m - 1)!) - m + 1.
"""
import ctypes
import os
import subprocess
from math import comb, factorial

import numpy as np

from .algebra import MonomialIndex, poly_powers, berkowitz_charpoly, add_exp, sub_exp
from .cohomology import (Hypersurface, cohomology_basis, hodge_count, is_smooth,
                         is_S_smooth, full_S, Section, affine_parts, FinalReduction)
from .policies import tweak, play, GameLog
from .precision import Precision, vp_factorial, hodge_polygon

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def build_helper():
    """Compile oracle/horner.c into oracle/_horner.so (plain gcc)."""
    src = os.path.join(_HERE, "horner.c")
    out = os.path.join(_HERE, "_horner.so")
    if not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", out, src])
    return out


def _helper():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build_helper())
        lib.oracle_horner_chunk.restype = ctypes.c_int
        lib.oracle_horner_chunk.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
            ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_int64),
            ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_uint64), ctypes.c_uint64]
        lib.oracle_matmul_mod.restype = None
        lib.oracle_matmul_mod.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64),
            ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64), ctypes.c_uint64]
        _LIB = lib
    return _LIB


def horner_python(A, B, W, k, q):
    """Algorithm 2: W <- M(0) M(1) ... M(k-1) W with M(y) = y A + B, mod q."""
    M = ((k - 1) * A + B) % q
    for _ in range(k):
        W = M.dot(W) % q
        M = (M - A) % q
    return W


_U64_CACHE = {}


def _parts_u64(parts):
    key = id(parts)
    hit = _U64_CACHE.get(key)
    if hit is None or hit[0] is not parts:
        hit = (parts, np.ascontiguousarray(
            np.stack([np.array(a, dtype=np.uint64) for a in parts])))
        _U64_CACHE[key] = hit
    return hit[1]


def horner_chunk(parts, x, v, k, W, q, use_c=True):
    """One chunk: A = sum v_i A_i, B = sum x_i A_i + A_{n+1}, then Algorithm 2."""
    n1 = len(x)
    s = parts[0].shape[0]
    c = W.shape[1]
    if use_c and q < (1 << 63):
        lib = _helper()
        P = _parts_u64(parts)
        Wa = np.ascontiguousarray(np.array(W, dtype=np.uint64))
        xa = np.array(x, dtype=np.int64)
        va = np.array(v, dtype=np.int64)
        rc = lib.oracle_horner_chunk(
            n1, s, c, k, P.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
            xa.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
            va.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
            Wa.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), q)
        if rc:
            raise MemoryError("oracle helper allocation failed")
        return Wa.astype(object)
    A = sum(v[i] * parts[i] for i in range(n1)) % q
    B = (sum(x[i] * parts[i] for i in range(n1)) + parts[n1]) % q
    return horner_python(A, B, W, k, q)


def D_coeff(j, m, N):
    """D_{j,m} = sum_{i=j}^{N-1} (-1)^{i+j} C(-m, i) C(i, j) (Prop. 2.1; summation index i)."""
    tot = 0
    for i in range(j, N):
        binom_neg = (-1) ** i * comb(m + i - 1, i)     # C(-m, i)
        tot += (-1) ** (i + j) * binom_neg * comb(i, j)
    return tot


class ZetaResult:
    pass


def frobenius_terms(X, basis, prec, S=None):
    """Prop. 2.1 terms for every basis column, Tweak'd and scaled.

    Yields (col, U, J, coefficient mod q) where the term is
      coefficient * x^U x^J / (x^S f^{p(m+j)}),
    coefficient = (D_{j,m} C_{j,alpha} mod p^{s_m}) * (p s_m - 1)! / (p(m+j) - 1)!,
    the factor p^{m-1} of Prop. 2.1 left out (restored in the normalisation).
    The numerator of Prop. 2.1 is x^{p(beta+alpha+1) - 1}; over x^S it is
    x^gamma with gamma = p(beta+alpha+1) - 1 + 1_S (p(beta+alpha+1) for S = {0..n}).
    """
    n, d, p, q = X.n, X.d, X.p, prec.q
    S = full_S(n) if S is None else S
    oneS = tuple(1 if i in S else 0 for i in range(X.nv))
    jmax = max(prec.N.values())
    powers = poly_powers(X.f, jmax - 1)
    for col, (m, beta) in enumerate(basis):
        N, s = prec.N[m], prec.s[m]
        ps = p ** s
        top = factorial(p * s - 1)
        for j in range(N):
            Djm = D_coeff(j, m, N)
            scale = (top // factorial(p * (m + j) - 1)) % q
            for alpha, Cja in powers[j].items():
                c = (Djm * Cja) % ps
                if c == 0:
                    continue
                gamma = tuple(p * (b + a + 1) - 1 + e for b, a, e in zip(beta, alpha, oneS))
                U, J = tweak(gamma, d * n - n)
                yield col, U, J, (c * scale) % q


def compute_zeta(n, d, p, coeffs, policy="depth_first", r=None, N=None,
                 column_order=None, use_c=True, want_P=True, normalise=True, S=None):
    """Run the whole computation.  Returns a ZetaResult with
    basis, prec (r, N_m, M, q), Y (unnormalised b x b mod q), C (columns of
    p^{m-n-1} sigma mod p^r), F (= C diag(p^{n-m})), P (list a_0..a_b) and
    the game log of the policy.

    S: the index set of Prop. 3.3 (default {0..n}); f must be S-smooth and
    d >= |S|.  Y depends on neither S nor the policy (module docstring)."""
    S = full_S(n) if S is None else tuple(sorted(set(S)))
    if not is_smooth(n, d, p, coeffs):
        raise ValueError("f is not smooth")
    if len(S) > d:
        raise ValueError("Prop. 3.3 needs d >= |S|")
    if S != full_S(n) and not is_S_smooth(n, d, p, coeffs, S):
        raise ValueError("f is not S-smooth")
    X = Hypersurface(n, d, p, coeffs)
    basis = cohomology_basis(X)
    b = len(basis)
    assert b == hodge_count(n, d)
    pole_orders = [m for m, _ in basis]
    prec = Precision(n, d, p, pole_orders, r=r, N=N)
    q = prec.q
    Sidx = MonomialIndex(X.nv, d * n - n)
    s = len(Sidx)

    # Steps 3-4: terms combined by U into s x b blocks.
    blocks = {}
    for col, U, J, c in frobenius_terms(X, basis, prec, S):
        if U not in blocks:
            blocks[U] = np.zeros((s, b), dtype=object)
        blk = blocks[U]
        blk[Sidx.pos[J], col] = (blk[Sidx.pos[J], col] + c) % q
    terms = list(blocks.items())

    # Step 5: the policy plays the game; chunks run Algorithm 2.
    sec = Section(X, q, column_order=column_order, S=S)
    parts_cache = {}
    log = GameLog()
    oneS = tuple(1 if i in S else 0 for i in range(X.nv))

    def reduce_chunk(u, v, k, w):
        # invariant: x^u g / x^S is a polynomial, so g has no monomial mu with
        # u_i + mu_i = 0 for i in S; those rows must be zero.
        zeros = tuple(i for i in S if u[i] == 0)
        if zeros:
            for row, mu in enumerate(Sidx.mons):
                if any(mu[i] == 0 for i in zeros):
                    assert not any(w[row]), "invalid monomial carries a coefficient"
        if v not in parts_cache:
            parts_cache[v] = affine_parts(X, sec, Sidx, v)
        x = tuple(ui - k * vi for ui, vi in zip(u, v))
        log.chunks += 1
        log.steps += k
        log.column_steps += k * int(sum(1 for c in range(b) if any(w[:, c])))
        return horner_chunk(parts_cache[v], x, v, k, w, q, use_c=use_c)

    def add(a, w):
        return (a + w) % q

    final = play(policy, terms, n, d, p, S, reduce_chunk, add, log)

    # Step 6: numerators x^u g / x^S at pole order n, summed per column.
    fin = FinalReduction(X, basis, q)
    Y = np.zeros((b, b), dtype=object)
    H = [dict() for _ in range(b)]
    for u, w in final:
        assert sum(u) == len(S) - 1
        for row, mu in enumerate(Sidx.mons):
            e = sub_exp(add_exp(u, mu), oneS)
            for col in range(b):
                a = w[row, col]
                if a:
                    assert min(e) >= 0
                    H[col][e] = (H[col].get(e, 0) + a) % q
    for col in range(b):
        Y[:, col] = fin.reduce(H[col])
    if not normalise:
        res = ZetaResult()
        res.n, res.d, res.p, res.coeffs = n, d, p, list(coeffs)
        res.basis, res.prec, res.Y, res.log, res.policy = basis, prec, Y, log, policy
        res.S = S
        return res

    # Step 7: normalisation.  Y = ((p s_m - 1)!/(n-1)!) p^{1-m} c, c known mod p^{r_m}.
    C = np.zeros((b, b), dtype=object)
    for col, (m, beta) in enumerate(basis):
        pr = p ** prec.r[m]
        sm = prec.s[m]
        v = vp_factorial(p * sm - 1, p)
        e = v - m + 1
        unit = (factorial(p * sm - 1) // p ** v) % q
        for row in range(b):
            y = int(Y[row, col])
            if e > 0:
                if y % (p ** e):
                    raise ArithmeticError("column %d not divisible by p^%d" % (col, e))
                z = y // (p ** e)
            else:
                z = y * p ** (-e)
            c = z * factorial(n - 1) * pow(unit, -1, q)
            C[row, col] = c % pr
    F = np.zeros((b, b), dtype=object)
    for col, (m, _) in enumerate(basis):
        F[:, col] = C[:, col] * p ** (n - m)

    res = ZetaResult()
    res.n, res.d, res.p, res.coeffs = n, d, p, list(coeffs)
    res.basis, res.prec, res.Y, res.C, res.F, res.log = basis, prec, Y, C, F, log
    res.policy = policy
    res.S = S
    if want_P:
        res.P, res.eps = charpoly_lift(n, p, F, C, pole_orders, prec)
    return res


def charpoly_lift(n, p, F, C, pole_orders, prec):
    """P(T) = det(1 - T F) in Z[T] (Sec. 2.1) from F known to the stated precision.

    With the columns of pole order m known mod p^{r_m + n - m}, a_i for
    i <= b/2 is known mod p^{e_i} (oracle.precision) and lifted to the
    symmetric range; the rest follows from the functional equation
    a_{b-i} = eps p^{w(b/2 - i)} a_i, w = n - 1, with
    eps = (-1)^b det(C) (a_b = (-1)^b det F and det F = det(C) p^{H(b)}).
    """
    b = len(pole_orders)
    w = n - 1
    cp = berkowitz_charpoly(F.tolist())   # det(T I - F) = sum cp[i] T^{b-i}; a_i = cp[i]
    a = [0] * (b + 1)
    a[0] = 1
    for i in range(1, b // 2 + 1):
        mod = p ** prec.e[i]
        x = cp[i] % mod
        if x > mod // 2:
            x -= mod
        a[i] = x
    rmin = min(prec.r.values())
    detC = berkowitz_charpoly(C.tolist())[b] * (-1) ** b   # det(C)
    sgn = ((-1) ** b * detC) % (p ** rmin)
    if sgn == 1:
        eps = 1
    elif sgn == p ** rmin - 1:
        eps = -1
    else:
        raise ArithmeticError("det(C) is not +-1 mod p^r: %d" % sgn)
    for i in range(0, (b + 1) // 2):
        j = b - i
        if j <= b // 2:
            continue
        a[j] = eps * p ** (w * (b - 2 * i) // 2) * a[i]
    return a, eps
