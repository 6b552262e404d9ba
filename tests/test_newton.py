"""Newton polygons and the p-rank filter of the Newton-strata search (host logic, against closed forms)."""
from fractions import Fraction

import zeta_inputs as zi
from oracle import cohomology, zeta as ozeta
from paper_2602_24155_gb300.newton import (newton_slopes, polygon_label, random_hypersurfaces, unit_roots_mod_p,
                                           vp)


def test_valuation():
    assert vp(7 ** 5 * 3, 7) == 5 and vp(-49, 7) == 2 and vp(13, 7) == 0


def test_elliptic_curves():
    # ordinary: 1 - aT + pT^2 with p not dividing a; supersingular: a = 0
    assert newton_slopes([1, -3, 7], 7) == [0, 1]
    assert newton_slopes([1, 0, 7], 7) == [Fraction(1, 2)] * 2
    assert newton_slopes([1, 7, 7], 7) == [Fraction(1, 2)] * 2   # p | a still supersingular (v(a) >= 1/2 line)


def test_products_of_polygons():
    # (1 + pT^2)^3: all slopes 1/2;  (1 - T)(1 - p^2 T): slopes 0 and 2 (weight 2)
    p = 11
    P = [1, 0, 3 * p, 0, 3 * p * p, 0, p ** 3]
    assert newton_slopes(P, p) == [Fraction(1, 2)] * 6
    assert polygon_label(newton_slopes([1, -(1 + p * p), p * p], p)) == "0^1 2^1"
    # a genus-2 curve of p-rank 1: (1 - aT + pT^2)(1 + pT^2) with p not dividing a
    a = 2
    P2 = [1, -a, 2 * p, -a * p, p * p]
    assert polygon_label(newton_slopes(P2, p)) == "0^1 1/2^2 1^1"
    assert unit_roots_mod_p(P2, p) == 1


def test_random_hypersurfaces_are_seeded():
    a = random_hypersurfaces(2, 5, 7, 3, seed=4)
    assert a == random_hypersurfaces(2, 5, 7, 3, seed=4)
    assert a != random_hypersurfaces(2, 5, 7, 3, seed=5)
    assert all(len(x[3]) == 21 and all(0 <= v < 7 for v in x[3]) for x in a)


def test_filter_precision_gives_p_mod_p_on_the_oracle():
    # a non-ordinary plane quintic over F_7: the r = 1 truncation gives P mod p, whose degree is the number of
    # slope-0 segments of the full Newton polygon
    n, d, p, c, _ = zi.draw_instance("quintic_curves", 12, cohomology.is_smooth)
    low = ozeta.compute_zeta(n, d, p, c, r=1)
    full = ozeta.compute_zeta(n, d, p, c)
    assert [a % p for a in low.P] == [a % p for a in full.P]
    slopes = newton_slopes(full.P, p)
    assert unit_roots_mod_p(low.P, p) == slopes.count(0) == 5
    assert polygon_label(slopes) == "0^5 1/2^2 1^5"


def test_k3_height_rule_on_synthetic_polygons():
    from paper_2602_24155_gb300.newton import k3_height
    p = 7
    # height 1: a_1 a unit; height 2: v(a_1) >= 1, v(a_2) = 1; supersingular: v(a_i) >= i
    base = [1] + [p ** i for i in range(1, 22)]
    h1 = list(base); h1[1] = 3
    h2 = list(base); h2[2] = 5 * p
    h3 = list(base); h3[3] = 2 * p * p
    assert k3_height(h1, p) == 1 and k3_height(h2, p) == 2 and k3_height(h3, p) == 3
    assert k3_height(base, p) is None


def test_k3_heights_at_precision_one_on_the_oracle():
    # Fermat quartic surface: supersingular for p = 3 mod 4; a random K3 whose a_1 vanishes mod p (Hasse-Witt, an
    # independent computation) has height >= 2
    from oracle import pins
    from paper_2602_24155_gb300.newton import k3_height
    low = ozeta.compute_zeta(3, 4, 7, zi.fermat(3, 4), r=1)
    assert k3_height(low.P, 7) is None
    n, d, p, c, _ = zi.draw_instance("quartic_k3", 12, cohomology.is_smooth)
    assert p == 7 and pins.hasse_witt_charpoly_mod_p(n, d, p, c)[1] % p == 0
    low = ozeta.compute_zeta(n, d, p, c, r=1)
    assert low.P[1] % p == 0
    assert k3_height(low.P, p) >= 2


def test_hodge_numbers_and_first_slope():
    from paper_2602_24155_gb300.newton import hodge_numbers, first_slope
    from oracle.cohomology import hodge_count
    # plane quintic (g = 6), quartic K3, cubic surface, cubic threefold (0, 5, 5, 0), cubic fourfold (1, 20, 1)
    assert hodge_numbers(2, 5) == {1: 6, 2: 6} and first_slope(2, 5) == (0, 6)
    assert hodge_numbers(3, 4) == {1: 1, 2: 19, 3: 1} and first_slope(3, 4) == (0, 1)
    assert hodge_numbers(3, 3) == {1: 0, 2: 6, 3: 0} and first_slope(3, 3) == (1, 6)
    assert hodge_numbers(4, 3) == {1: 0, 2: 5, 3: 5, 4: 0} and first_slope(4, 3) == (1, 5)
    assert hodge_numbers(5, 3) == {1: 0, 2: 1, 3: 20, 4: 1, 5: 0} and first_slope(5, 3) == (1, 1)
    for n, d in [(2, 4), (2, 5), (3, 3), (3, 4), (3, 5), (4, 3), (5, 3)]:
        assert sum(hodge_numbers(n, d).values()) == hodge_count(n, d)


def test_first_slope_length_is_the_p_rank_for_curves_and_the_slope_one_length_for_threefolds():
    from random import Random
    from paper_2602_24155_gb300.newton import first_slope_length
    p = 7
    rng = Random(5)
    for _ in range(200):                       # h0 = 0: the degree of P mod p
        P = [1] + [rng.randrange(-500, 500) for _ in range(12)]
        assert first_slope_length(P, p, 0) == unit_roots_mod_p(P, p)
    # cubic threefold polygons (weight 3, b = 10, Hodge polygon H(i) = i for i <= 5, then slope 2): coefficients
    # with v_p(a_i) on a chosen polygon (units 2 and 3 are prime to p)
    H = [0] + list(range(1, 6)) + [5 + 2 * (i - 5) for i in range(6, 11)]
    ordinary = [1] + [2 * p ** H[i] for i in range(1, 11)]
    assert newton_slopes(ordinary, p) == [1] * 5 + [2] * 5
    assert first_slope_length(ordinary, p, 1) == 5
    almost = list(ordinary)
    almost[5] = 3 * p ** 6                     # v(a_5) = 6: slopes 1^4 (3/2)^2 2^4, almost ordinary
    assert newton_slopes(almost, p) == [1] * 4 + [Fraction(3, 2)] * 2 + [2] * 4
    assert first_slope_length(almost, p, 1) == 4
    lower = list(almost)
    lower[4] = 3 * p ** 5                      # v(a_4) = 5, v(a_6) = 8 as well: slopes 1^3 (3/2)^4 2^3
    lower[6] = 3 * p ** 8
    assert newton_slopes(lower, p) == [1] * 3 + [Fraction(3, 2)] * 4 + [2] * 3
    assert first_slope_length(lower, p, 1) == 3
    # the truncation of an r = 1 run (a_i known mod p^(1 + H(i))) gives the same answer
    for P in (ordinary, almost, lower):
        low = [a % p ** (1 + H[i]) for i, a in enumerate(P)]
        assert first_slope_length(low, p, 1) == first_slope_length(P, p, 1)


def test_fourfold_height_rule_and_hodge_polygon():
    """Cubic fourfolds: H(i) = 2i - 1 on 1..21 and 44 at 22 (Hodge numbers 1, 20, 1); the height is the least i with
    v(a_i) <= 2i - 1, decided by a_i mod p^(2i).  Synthetic polygons of heights 1, 2, 3 and a supersingular one, the
    Fermat cubic fourfold over F_7 (ordinary: p = 1 mod 3) from Weil's Gauss-sum formula, and the dense fourfold of
    tests/golden/cubic_fourfold_f7.txt whose a_1 = 0 and a_2 = -7^4 (point counts) rule out heights 1 and 2."""
    from oracle import pins
    from paper_2602_24155_gb300.newton import fourfold_height, hodge_polygon
    H = hodge_polygon(5, 3)
    assert H[:4] == [0, 1, 3, 5] and H[21] == 41 and H[22] == 44 and len(H) == 23
    assert hodge_polygon(3, 5)[4] == 0 and hodge_polygon(3, 5)[5] == 1 and hodge_polygon(3, 5)[52] == 52
    p = 7
    base = [1] + [p ** (2 * i) for i in range(1, 23)]    # every a_i of valuation 2i: no finite height <= 11
    h1 = list(base); h1[1] = 3 * p
    h2 = list(base); h2[2] = 5 * p ** 3
    h3 = list(base); h3[3] = 2 * p ** 5
    assert [fourfold_height(P, p) for P in (h1, h2, h3)] == [1, 2, 3]
    assert fourfold_height(base, p) is None
    assert fourfold_height(pins.fermat_charpoly(5, 3, 7), 7) == 1
    s1, s2 = 2801 - sum(p ** i for i in range(5)), 5889703 - sum(p ** (2 * i) for i in range(5))
    a1, a2 = -s1, (s1 * s1 - s2) // 2
    assert a1 == 0 and a2 == -p ** 4
    assert fourfold_height([1, a1, a2] + [0] * 20, p) != 1 and fourfold_height([1, a1, a2] + [0] * 20, p) != 2
