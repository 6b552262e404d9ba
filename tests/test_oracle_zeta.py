"""End-to-end pins of the oracle: P(T) against point counts, closed forms and Weil's theorems."""
import os

import numpy as np
import pytest

import zeta_inputs as zi
from oracle import cohomology, pins, zeta
from oracle.precision import hodge_polygon

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _instance(workload, i):
    n, d, p, c, _ = zi.draw_instance(workload, i, cohomology.is_smooth)
    return n, d, p, c


@pytest.fixture(scope="module")
def quartic_f11():
    n, d, p, c = _instance("quartic_curve_f11", 0)
    return (n, d, p, c), zeta.compute_zeta(n, d, p, c)


def test_quartic_f11_matches_brute_force_counts(quartic_f11):
    (n, d, p, c), res = quartic_f11
    counts = [pins.count_points(n, d, p, c, r) for r in (1, 2, 3)]
    # genus 3: a_1..a_3 fix P(T) through the functional equation
    assert res.P[:4] == pins.counts_to_charpoly_prefix(n, p, counts)
    assert pins.charpoly_to_counts(n, p, res.P, 3) == counts


def test_quartic_f11_golden(quartic_f11):
    # stored by tests/golden/make_golden.py from the oracle after the counts above pinned it
    (n, d, p, c), res = quartic_f11
    with open(os.path.join(GOLDEN, "quartic_curve_f11.txt")) as fh:
        lines = dict(l.split(":", 1) for l in fh.read().strip().splitlines() if ":" in l)
    assert [int(x) for x in lines["coeffs"].split()] == c
    assert [int(x) for x in lines["P"].split()] == res.P


@pytest.mark.parametrize("p", [7, 13])
def test_random_quartics_match_counts(p):
    # several random smooth quartics: a_1..a_3 determine P
    for seed in range(2):
        att = 0
        while True:
            c = zi.dense_candidate(2, 4, p, 100 + seed, p, att)
            att += 1
            if cohomology.is_smooth(2, 4, p, c):
                break
        res = zeta.compute_zeta(2, 4, p, c)
        counts = [pins.count_points(2, 4, p, c, r) for r in (1, 2, 3)]
        assert res.P[:4] == pins.counts_to_charpoly_prefix(2, p, counts)


def test_quintic_curve_f7_matches_counts_and_hasse_witt():
    n, d, p, c = _instance("quintic_curves", 0)
    assert p == 7
    res = zeta.compute_zeta(n, d, p, c)
    counts = [pins.count_points(n, d, p, c, r) for r in (1, 2, 3)]
    assert res.P[:4] == pins.counts_to_charpoly_prefix(n, p, counts)
    hw = pins.hasse_witt_charpoly_mod_p(n, d, p, c)
    assert [a % p for a in res.P[:len(hw)]] == hw
    assert all(a % p == 0 for a in res.P[len(hw):])
    _weil_checks(res)


@pytest.mark.parametrize("n,d,p", [(2, 4, 13), (2, 5, 11), (2, 4, 17)])
def test_fermat_curves_gauss_sum_closed_form(n, d, p):
    res = zeta.compute_zeta(n, d, p, zi.fermat(n, d))
    assert res.P == pins.fermat_charpoly(n, d, p)


def test_hasse_witt_on_random_curves():
    for i in (1, 2, 3):
        n, d, p, c = _instance("quintic_curves", i)
        if p > 13:
            continue
        res = zeta.compute_zeta(n, d, p, c)
        hw = pins.hasse_witt_charpoly_mod_p(n, d, p, c)
        assert [a % p for a in res.P[:len(hw)]] == hw
        _weil_checks(res)


def _weil_checks(res):
    n, p = res.n, res.p
    pole = [m for m, _ in res.basis]
    P = res.P
    b = len(P) - 1
    assert P[0] == 1
    assert pins.root_moduli_ok(n, p, P)
    assert pins.newton_above_hodge(n, p, P, pole)
    # the upper coefficients computed directly agree with the functional equation
    from oracle.algebra import berkowitz_charpoly
    cp = berkowitz_charpoly(res.F.tolist())
    H = hodge_polygon(n, pole)
    rmin = min(res.prec.r.values())
    for j in range(b // 2 + 1, b + 1):
        mod = p ** (rmin + H[j])
        assert (cp[j] - P[j]) % mod == 0


def test_weil_invariants_quartic(quartic_f11):
    _, res = quartic_f11
    _weil_checks(res)


def test_policies_give_identical_unnormalised_columns(quartic_f11):
    # Y depends only on B, N_m and M: every policy plays to the same classes (Sec. 3.4)
    (n, d, p, c), ref = quartic_f11
    for policy in ("p_chunk", "var_by_var"):
        res = zeta.compute_zeta(n, d, p, c, policy=policy, want_P=False)
        assert (res.Y == ref.Y).all()
        assert res.log.steps <= ref.log.steps


def test_section_choice_does_not_change_the_result(quartic_f11):
    # a different right inverse of the Jacobian map (columns visited in reverse)
    (n, d, p, c), ref = quartic_f11
    X = cohomology.Hypersurface(n, d, p, c)
    ncols = len(X.jacobian_matrix((n + 1) * (d - 2) + 1)[2])
    res = zeta.compute_zeta(n, d, p, c, column_order=list(range(ncols))[::-1], want_P=False)
    assert (res.Y == ref.Y).all()


def test_precision_is_stable_under_more_terms(quartic_f11):
    (n, d, p, c), ref = quartic_f11
    N = {m: k + 1 for m, k in ref.prec.N.items()}
    res = zeta.compute_zeta(n, d, p, c, N=N, r=ref.prec.r)
    for col, (m, _) in enumerate(ref.basis):
        assert ((res.C[:, col] - ref.C[:, col]) % p ** ref.prec.r[m] == 0).all()
    assert res.P == ref.P


def test_exact_divisibility_fails_for_a_planted_mistake(quartic_f11):
    # a dropped pre-scale (one term's factorial ratio) must break the p^v divisibility
    # or the result; checks that the invariant has teeth.
    (n, d, p, c), ref = quartic_f11
    orig = zeta.frobenius_terms

    def broken(X, basis, prec, S=None):
        for k, (col, U, J, val) in enumerate(orig(X, basis, prec, S)):
            yield col, U, J, (val * (1 if k % 7 else 2)) % prec.q
    zeta.frobenius_terms = broken
    try:
        try:
            res = zeta.compute_zeta(n, d, p, c)
            caught = res.P != ref.P
        except ArithmeticError:
            caught = True
    finally:
        zeta.frobenius_terms = orig
    assert caught


def test_gauss_sum_formula_against_brute_force_counts():
    # the closed form itself, checked by counting points of x^4 + y^4 + z^4 over F_13^r, r = 1..3
    P = pins.fermat_charpoly(2, 4, 13)
    counts = [pins.count_points(2, 4, 13, zi.fermat(2, 4), r) for r in (1, 2, 3)]
    assert pins.charpoly_to_counts(2, 13, P, 3) == counts


def test_hasse_witt_against_brute_force_counts():
    # P(T) mod p from the Hasse-Witt matrix against P(T) determined by point counts (genus 3, F_7)
    att = 0
    while True:
        c = zi.dense_candidate(2, 4, 7, 555, 0, att)
        att += 1
        if cohomology.is_smooth(2, 4, 7, c):
            break
    counts = [pins.count_points(2, 4, 7, c, r) for r in (1, 2, 3)]
    a = pins.counts_to_charpoly_prefix(2, 7, counts)
    hw = pins.hasse_witt_charpoly_mod_p(2, 4, 7, c)
    assert [x % 7 for x in a] == hw


def test_fermat_quintic_surface_over_f11_is_ordinary():
    # the paper's statement (Sec. 6, quintic surfaces) that x^5 + y^5 + z^5 + w^5 is ordinary at 11, from Weil's
    # Gauss-sum formula: degree 52, every reciprocal root of absolute value 11, Newton polygon = Hodge polygon
    # (slopes 0, 1, 2 with multiplicities 4, 44, 4)
    from oracle.precision import hodge_polygon, vp
    P = pins.fermat_charpoly(3, 5, 11, dps=200)
    assert len(P) == 53 and P[0] == 1
    assert pins.root_moduli_ok(3, 11, P, dps=200)
    H = hodge_polygon(3, [1] * 4 + [2] * 44 + [3] * 4)
    assert all(P[i] != 0 and vp(P[i], 11) == H[i] for i in range(1, 53))
