"""Pins of the oracle's building blocks against closed forms and library routines."""
import random
from math import comb

import numpy as np
import pytest

import zeta_inputs as zi
from oracle import algebra, cohomology, policies, precision, zeta


def test_monomial_order_and_count():
    assert algebra.monomials(3, 2) == [(2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2)]
    for nv in range(1, 6):
        for deg in range(0, 9):
            ms = algebra.monomials(nv, deg)
            assert len(ms) == comb(deg + nv - 1, nv - 1)
            assert ms == sorted(ms, reverse=True)
    assert algebra.monomials(3, -1) == []


def test_berkowitz_matches_numpy_on_random_integer_matrices():
    rng = random.Random(5)
    for b in range(1, 8):
        F = [[rng.randint(-4, 4) for _ in range(b)] for _ in range(b)]
        cp = algebra.berkowitz_charpoly(F)
        ref = np.poly(np.array(F, dtype=float))
        assert np.allclose(cp, ref, atol=1e-6 * max(1, np.abs(ref).max()))


def test_berkowitz_companion_closed_form():
    # companion matrix of T^4 - 3T^3 + 5T - 7 has that characteristic polynomial
    coeffs = [1, -3, 0, 5, -7]
    b = 4
    Cm = [[0] * b for _ in range(b)]
    for i in range(1, b):
        Cm[i][i - 1] = 1
    for i in range(b):
        Cm[i][b - 1] = -coeffs[b - i]
    assert algebra.berkowitz_charpoly(Cm) == coeffs


@pytest.mark.parametrize("k", [5, 30])
def test_right_inverse_mod_prime_power(k):
    # k = 5 runs the int64 elimination, k = 30 (q^2 > 2^62) the Python-integer one
    rng = random.Random(2)
    p = 7
    q = p ** k
    for _ in range(5):
        M = [[rng.randrange(q) for _ in range(9)] for _ in range(5)]
        X, piv = algebra.right_inverse_mod(M, q, p)
        prod = np.array(M, dtype=object).dot(X) % q
        assert (prod == np.eye(5, dtype=int).astype(object)).all()


def test_tweak_front_and_examples():
    # Alg. 1 removes units from the lowest index first
    assert policies.tweak((3, 4, 5), 5) == ((0, 2, 5), (3, 2, 0))
    assert policies.tweak((0, 0, 9), 4) == ((0, 0, 5), (0, 0, 4))
    rng = random.Random(1)
    for _ in range(200):
        I = tuple(rng.randint(0, 6) for _ in range(4))
        m = rng.randint(0, 10)
        u, J = policies.tweak(I, m)
        assert tuple(a + b for a, b in zip(u, J)) == I
        assert sum(J) == min(m, sum(I))
        # everything before the last touched index is exhausted
        touched = [i for i in range(4) if J[i]]
        if touched:
            assert all(u[i] == 0 for i in range(touched[-1]))


def test_greedy_direction_properties():
    rng = random.Random(3)
    for _ in range(500):
        n = rng.choice([2, 3])
        d = rng.choice([n + 1, n + 2])
        u = tuple(rng.randint(0, 9) for _ in range(n + 1))
        if sum(u) < d:
            continue
        S = set(range(n + 1))
        v = policies.greedy_v(d, u, S)
        assert sum(v) == d
        assert all(0 <= v[i] <= u[i] for i in range(n + 1))
        assert all(v[i] > 0 for i in range(n + 1) if u[i] > 0)
    # a worked case: S first gives (1,1,1), then round robin from index 0
    assert policies.greedy_v(5, (13, 7, 7), {0, 1, 2}) == (2, 2, 1)


def test_k_max_definition():
    # largest k with u - k v >= 0 and |u - k v| >= n
    assert policies.k_max((10, 6, 6), (2, 2, 1), 2, 5) == 3
    assert policies.k_max((4, 4, 4), (2, 2, 1), 2, 5) == 2


def test_hodge_count_matches_basis_size_and_hodge_numbers():
    # (n, d) -> b and the per-pole-order counts (genus 3, genus 6, K3 (1,19,1))
    cases = {(2, 4): [3, 3], (2, 5): [6, 6], (3, 4): [1, 19, 1]}
    for (n, d), per_m in cases.items():
        p = 7 if d != 7 else 11
        _, _, _, c, _ = zi.draw_instance({(2, 4): "quartic_curve_f11", (2, 5): "quintic_curves",
                                          (3, 4): "quartic_k3"}[(n, d)], 0, cohomology.is_smooth)
        p = zi.instance_shape({(2, 4): "quartic_curve_f11", (2, 5): "quintic_curves",
                               (3, 4): "quartic_k3"}[(n, d)], 0)[2]
        X = cohomology.Hypersurface(n, d, p, c)
        basis = cohomology.cohomology_basis(X)
        assert len(basis) == cohomology.hodge_count(n, d) == sum(per_m)
        assert [sum(1 for m, _ in basis if m == mm) for mm in range(1, n + 1)] == per_m


def test_smoothness_test():
    # Fermat curves and surfaces are smooth for p not dividing d
    for (n, d, p) in [(2, 4, 7), (2, 5, 11), (3, 4, 13)]:
        assert cohomology.is_smooth(n, d, p, zi.fermat(n, d))
    # a curve with a rational singular point at [0:0:1] (no monomial of z-degree >= d-1)
    rng = random.Random(4)
    for _ in range(5):
        mons = algebra.monomials(3, 4)
        c = [0 if m[2] >= 3 else rng.randrange(11) for m in mons]
        assert not cohomology.is_smooth(2, 4, 11, c)
    # the cone x^2 + y^2 over a point... x^d + y^d is singular in P^2 at [0:0:1]
    c = [1 if m in [(4, 0, 0), (0, 4, 0)] else 0 for m in algebra.monomials(3, 4)]
    assert not cohomology.is_smooth(2, 4, 7, c)


def _quartic():
    n, d, p, c, _ = zi.draw_instance("quartic_curve_f11", 0, cohomology.is_smooth)
    return n, d, p, c


def test_section_identity_and_R_affine():
    n, d, p, c = _quartic()
    q = p ** 6
    X = cohomology.Hypersurface(n, d, p, c)
    sec = cohomology.Section(X, q)
    kappa = (n + 1) * (d - 2) + 1
    for gamma in algebra.monomials(n + 1, kappa):
        g = sec.solve(gamma)
        tot = {}
        for i in range(n + 1):
            for e, a in algebra.poly_mul(g[i], X.df[i]).items():
                tot[e] = (tot.get(e, 0) + a) % q
        tot = {e: a for e, a in tot.items() if a}
        assert tot == {gamma: 1}
    Sidx = algebra.MonomialIndex(n + 1, d * n - n)
    v = (2, 1, 1)
    R = [cohomology.R_matrix(X, sec, Sidx, (t, 2 * t, 5), v) for t in range(3)]
    assert ((R[2] - 2 * R[1] + R[0]) % q == 0).all()
    parts = cohomology.affine_parts(X, sec, Sidx, v)
    u = (3, 4, 5)
    lhs = cohomology.R_matrix(X, sec, Sidx, u, v)
    rhs = (sum(u[i] * parts[i] for i in range(3)) + parts[3]) % q
    assert (lhs == rhs).all()


def test_horner_is_the_explicit_product_and_c_matches_python():
    rng = random.Random(7)
    for q in [7 ** 5, 11 ** 14, 47 ** 11]:
        s, c = 6, 3
        parts = [np.array([[rng.randrange(q) for _ in range(s)] for _ in range(s)], dtype=object)
                 for _ in range(4)]
        x, v, k = (3, 1, 2), (2, 2, 1), 4
        W = np.array([[rng.randrange(q) for _ in range(c)] for _ in range(s)], dtype=object)
        # explicit product M(0) M(1) ... M(k-1) W with M(y) = R_{x + y v}
        ref = W.copy()
        for y in range(k - 1, -1, -1):
            u = tuple(a + y * b for a, b in zip(x, v))
            My = (sum(u[i] * parts[i] for i in range(3)) + parts[3]) % q
            ref = My.dot(ref) % q
        py = zeta.horner_chunk(parts, x, v, k, W, q, use_c=False)
        cc = zeta.horner_chunk(parts, x, v, k, W, q, use_c=True)
        assert (py == ref).all()
        assert (cc == ref).all()


def test_precision_rules():
    # Legendre's formula against a direct factorial valuation
    from math import factorial
    for p in [7, 11]:
        for x in [1, 6, 7, 48, 49, 50, 120]:
            assert precision.vp_factorial(x, p) == (precision.vp(factorial(x), p) if x > 0 else 0)
    # genus 3 over F_11: a_3 <= 20 * 11^1.5 ~ 730, 2*730 < 11^4; columns of pole order 1
    # carry a factor p in every minor they enter, so they need one digit less
    assert precision.coefficient_digits(2, 11, 6) == [1, 2, 3, 4]
    assert precision.relative_precisions(2, 11, [1, 1, 1, 2, 2, 2]) == {1: 3, 2: 4}
    # genus 6 over F_41: 2 * C(12,6) * 41^3 > 41^5, so e_6 = 6 and r_2 = 6, r_1 = 5
    assert precision.relative_precisions(2, 41, [1] * 6 + [2] * 6) == {1: 5, 2: 6}
    # K3 (Hodge slopes 2, 1 x 19, 0) over F_7
    pr = precision.Precision(3, 4, 7, [1] + [2] * 19 + [3])
    assert pr.r[3] >= pr.r[2] >= pr.r[1] >= 1
    # series orders reproduce the smallest stable N found for plane curves
    assert precision.series_order(1, 4, 2, 11) == 5
    assert precision.series_order(2, 4, 2, 11) == 4
    assert precision.series_order(1, 7, 2, 7) == 9
    assert precision.series_order(2, 7, 2, 7) == 8


def test_D_coefficients_recombine_the_binomial_series():
    # sum_j D_{j,m} y^j equals sum_{i<N} C(-m,i) (y-1)^i (Prop. 2.1 with y = sigma(f)/f^p)
    import sympy
    y = sympy.symbols('y')
    for m in (1, 2, 3):
        for N in (1, 3, 5):
            lhs = sum(zeta.D_coeff(j, m, N) * y ** j for j in range(N))
            rhs = sum(sympy.binomial(-m, i) * (y - 1) ** i for i in range(N))
            assert sympy.expand(lhs - rhs) == 0


def test_weil_root_check_with_repeated_roots():
    # products of (1 - alpha T) with known reciprocal roots: repeated roots of modulus p pass, one root of
    # another modulus fails; the square-free part keeps each distinct root once
    from numpy.polynomial import polynomial as npoly
    from oracle import pins

    def prod(factors):
        P = [1]
        for f in factors:
            P = [int(x) for x in npoly.polymul(P, f)]
        return P
    P = prod([[1, -7], [1, -7], [1, 7], [1, 0, -49], [1, 0, 49]])   # roots 7, 7, -7, +-7, +-7i
    assert pins.root_moduli_ok(3, 7, P)
    Q = pins._squarefree_part(P)
    assert len(Q) - 1 == 4                                            # 7, -7, 7i, -7i
    assert not pins.root_moduli_ok(3, 7, prod([[1, -7], [1, -7], [1, -5]]))
    assert not pins.root_moduli_ok(3, 7, prod([[1, 0, -49], [1, -8]]))
