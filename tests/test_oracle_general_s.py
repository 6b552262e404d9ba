"""General S in Prop. 3.3 (oracle): S-smoothness, the section of J_S and R_{u,v} for S other than {0..n}.

Pins that do not go through the formulas under test:
  - S-smoothness (Definition 3.1) against common zeros that can be read off the coefficients;
  - the section against the polynomial identity it must satisfy;
  - R_{u,v} against the printed two-sum formula of Prop. 3.3, evaluated with polynomial arithmetic;
  - for curves, where S = {0..n} also applies, the unnormalised columns Y are the coordinates of one
    truncated Frobenius expansion, so they must equal those of the S = {0..n} path for every S and policy;
  - cubic surfaces (d = 3 < n + 1, so only a smaller S applies) against the Gauss-sum closed form of the
    Fermat surface and against brute-force point counts over F_p and F_{p^2}.
"""
import os

import numpy as np
import pytest

import zeta_inputs as zi
from oracle import algebra, cohomology, pins, zeta
from oracle.algebra import add_exp, sub_exp, poly_add, poly_scale, poly_deriv, poly_times_monomial


def _draw(n, d, p, seed, S, skip=0):
    """Seeded dense f that is smooth and S-smooth (the `skip`-th such draw)."""
    att = 0
    found = 0
    while True:
        c = zi.dense_candidate(n, d, p, seed, p, att)
        att += 1
        if cohomology.is_smooth(n, d, p, c) and cohomology.is_S_smooth(n, d, p, c, S):
            if found == skip:
                return c
            found += 1


def _mon_index(nv, d, mono):
    return algebra.monomials(nv, d).index(mono)


def test_S_smoothness_follows_definition():
    # S = {0..n} is smoothness itself
    for att in range(6):
        c = zi.dense_candidate(2, 4, 7, 3, 0, att)
        assert cohomology.is_S_smooth(2, 4, 7, c, (0, 1, 2)) == cohomology.is_smooth(2, 4, 7, c)
    # x0^4 + x1^4 is singular at (0:0:1): neither smooth nor S-smooth for any S
    c = [0] * 15
    c[_mon_index(3, 4, (4, 0, 0))] = 1
    c[_mon_index(3, 4, (0, 4, 0))] = 1
    assert not cohomology.is_smooth(2, 4, 7, c)
    assert not cohomology.is_S_smooth(2, 4, 7, c, (2,))
    # Fermat hypersurfaces: J_{n} = <x_n^{d-1}, x_i^d (i < n)> has no common zero
    for n, d, p in [(2, 4, 11), (3, 3, 7), (3, 4, 7)]:
        assert cohomology.is_S_smooth(n, d, p, zi.fermat(n, d), (n,))
    # With no x_n^d term, (0:...:0:1) is a common zero of d_n f and every x_i d_i f (i < n):
    # smooth surfaces and curves with that coefficient zero are not {n}-smooth
    for n, d, p in [(2, 4, 11), (3, 3, 7)]:
        tested = 0
        for att in range(60):
            c = zi.dense_candidate(n, d, p, 4, 1, att)
            c[_mon_index(n + 1, d, (0,) * n + (d,))] = 0
            if cohomology.is_smooth(n, d, p, c):
                assert not cohomology.is_S_smooth(n, d, p, c, (n,))
                tested += 1
        assert tested >= 5


def test_compute_zeta_refuses_what_prop_3_3_excludes():
    c = _draw(3, 3, 7, 8, (3,))
    with pytest.raises(ValueError):
        zeta.compute_zeta(3, 3, 7, c, S=(0, 1, 2, 3))      # d < |S|
    bad = zi.fermat(2, 4)
    bad[_mon_index(3, 4, (0, 0, 4))] = 0
    bad[_mon_index(3, 4, (1, 0, 3))] = 1                    # x0^4 + x1^4 + x0 x2^3: smooth, not {2}-smooth
    assert cohomology.is_smooth(2, 4, 11, bad)
    with pytest.raises(ValueError):
        zeta.compute_zeta(2, 4, 11, bad, S=(2,))


@pytest.mark.parametrize("n,d,p,S", [(3, 3, 7, (3,)), (2, 4, 11, (2,)), (2, 4, 7, (0, 2))])
def test_section_of_J_S_solves_the_identity(n, d, p, S):
    c = _draw(n, d, p, 9, S)
    q = p ** 5
    X = cohomology.Hypersurface(n, d, p, c)
    sec = cohomology.Section(X, q, S=S)
    kappa = cohomology.kappa_S(n, d, S)
    assert kappa == d + d * n - n - len(S)
    for gamma in algebra.monomials(n + 1, kappa):
        G = sec.solve(gamma)
        tot = {}
        for i in range(n + 1):
            if i not in S:
                assert all(nu[i] >= 1 for nu in G[i])            # G_i = x_i g_i
            for e, a in algebra.poly_mul(G[i], X.df[i]).items():
                tot[e] = (tot.get(e, 0) + a) % q
        assert {e: a for e, a in tot.items() if a} == {gamma: 1}


def _printed_R(X, sec, Sidx, u, v):
    """Prop. 3.3 as printed: g_i from x^v g / x^S = sum_{i in S} g_i d_i f + sum_{i not in S} x_i g_i d_i f,
    R(g) = x^S (sum_{i in S} (u_i g_i + x_i d_i g_i) / x_i + sum_{i not in S} ((u_i + 1) g_i + x_i d_i g_i))."""
    q, nv, S = sec.q, X.nv, sec.S
    oneS = tuple(1 if i in S else 0 for i in range(nv))
    R = np.zeros((len(Sidx), len(Sidx)), dtype=object)
    for col, mu in enumerate(Sidx.mons):
        gamma = sub_exp(add_exp(v, mu), oneS)
        if min(gamma) < 0:
            continue
        G = sec.solve(gamma)
        out = {}
        for i in range(nv):
            ei = tuple(1 if t == i else 0 for t in range(nv))
            if i in S:
                g = G[i]
                h = poly_add(poly_scale(g, u[i]), poly_times_monomial(poly_deriv(g, i), ei))
                h = {add_exp(sub_exp(e, ei), oneS): a for e, a in h.items()}      # / x_i, then * x^S
            else:
                g = {sub_exp(nu, ei): a for nu, a in G[i].items()}
                h = poly_add(poly_scale(g, u[i] + 1), poly_times_monomial(poly_deriv(g, i), ei))
                h = {add_exp(e, oneS): a for e, a in h.items()}                    # * x^S
            out = poly_add(out, h)
        for e, a in out.items():
            R[Sidx.pos[e], col] = a % q
    return R


@pytest.mark.parametrize("n,d,p,S,v,u", [
    (3, 3, 7, (3,), (1, 0, 1, 1), (2, 3, 0, 4)),
    (3, 3, 7, (3,), (0, 0, 0, 3), (0, 1, 0, 5)),
    (2, 4, 11, (2,), (2, 1, 1), (3, 4, 5)),
    (2, 4, 11, (1, 2), (0, 2, 2), (0, 6, 2)),
])
def test_R_matrix_matches_printed_formula(n, d, p, S, v, u):
    c = _draw(n, d, p, 10, S)
    q = p ** 6
    X = cohomology.Hypersurface(n, d, p, c)
    sec = cohomology.Section(X, q, S=S)
    Sidx = algebra.MonomialIndex(n + 1, d * n - n)
    R = cohomology.R_matrix(X, sec, Sidx, u, v)
    assert (R == _printed_R(X, sec, Sidx, u, v)).all()
    parts = cohomology.affine_parts(X, sec, Sidx, v)
    assert (R == (sum(u[i] * parts[i] for i in range(n + 1)) + parts[n + 1]) % q).all()


@pytest.mark.parametrize("workload_or_p,S", [("quartic_curve_f11", (1, 2)), (7, (2,)), (7, (0, 2))])
def test_curves_Y_independent_of_S_and_policy(workload_or_p, S):
    if isinstance(workload_or_p, str):
        n, d, p, c, _ = zi.draw_instance(workload_or_p, 0, cohomology.is_smooth)
        assert cohomology.is_S_smooth(n, d, p, c, S)
    else:
        n, d, p = 2, 4, workload_or_p
        c = _draw(n, d, p, 11, S)
    ref = zeta.compute_zeta(n, d, p, c)
    for policy in ("depth_first", "p_chunk", "var_by_var"):
        res = zeta.compute_zeta(n, d, p, c, policy=policy, S=S)
        assert (res.Y == ref.Y).all(), policy
        assert res.P == ref.P


def test_k3_surface_Y_independent_of_S():
    # a quartic K3 surface (d = n + 1) admits S = {0..3} and S = {3}: at relative precision 1 (a truncated
    # expansion, the same form for both) the unnormalised columns must agree exactly
    n, d, p, c, _ = zi.draw_instance("quartic_k3", 1, cohomology.is_smooth)
    assert cohomology.is_S_smooth(n, d, p, c, (3,))
    a = zeta.compute_zeta(n, d, p, c, policy="p_chunk", r=1, want_P=False)
    b = zeta.compute_zeta(n, d, p, c, policy="p_chunk", r=1, want_P=False, S=(3,))
    assert (a.Y == b.Y).all()


@pytest.mark.parametrize("p", [7, 13])
def test_fermat_cubic_surface_closed_form(p):
    P = zeta.compute_zeta(3, 3, p, zi.fermat(3, 3), policy="p_chunk", S=(3,)).P
    assert P == pins.fermat_charpoly(3, 3, p)


@pytest.mark.parametrize("p", [7, 11])
def test_random_cubic_surfaces_match_counts(p):
    c = _draw(3, 3, p, 7, (3,))
    res = {pol: zeta.compute_zeta(3, 3, p, c, policy=pol, S=(3,)) for pol in ("depth_first", "p_chunk")}
    r = res["p_chunk"]
    assert (res["depth_first"].Y == r.Y).all()
    counts = [pins.count_points(3, 3, p, c, k) for k in (1, 2)]
    assert r.P[:3] == pins.counts_to_charpoly_prefix(3, p, counts)
    assert pins.charpoly_to_counts(3, p, r.P, 2) == counts
    assert pins.root_moduli_ok(3, p, r.P)
    assert pins.newton_above_hodge(3, p, r.P, [m for m, _ in r.basis])


@pytest.mark.skipif(not os.environ.get("ZETA_SLOW_ORACLE"), reason="about 13 minutes; set ZETA_SLOW_ORACLE=1")
def test_cubic_threefold_f11_precision_of_the_printed_modulus():
    """A dense cubic threefold over F_11 (S = {4}) at the series orders N = 3 (arithmetic mod 11^8, the precision the
    paper prints for this case) and N = 4 (mod 11^9).  Each further term adds one p-adic digit to the Frobenius
    columns: C agrees between the two mod p^2 (pole order 2) and p^3 (pole order 3) but not beyond, and det C is
    +-1 mod p^3 only at N = 3, so mod 11^8 does not give the relative precision the lift of P(T) needs.  The
    coefficients it does fix, a_1 and a_2 mod 11^4, equal those of brute-force counts over F_11 and F_121."""
    from oracle.algebra import berkowitz_charpoly
    n, d, p = 4, 3, 11
    att = 0
    while True:
        c = zi.dense_candidate(n, d, p, 11, 0, att)
        att += 1
        if cohomology.is_smooth(n, d, p, c) and cohomology.is_S_smooth(n, d, p, c, (4,)):
            break
    res = {N: zeta.compute_zeta(n, d, p, c, policy="p_chunk", S=(4,), N=N, want_P=False) for N in (3, 4)}
    assert res[3].prec.M == 8 and res[4].prec.M == 9
    for col, (m, _) in enumerate(res[3].basis):
        diff = [int(a) - int(b) for a, b in zip(res[3].C[:, col], res[4].C[:, col])]
        agree = m   # digits: 2 for pole order 2, 3 for pole order 3
        assert all(x % p ** agree == 0 for x in diff)
        assert any(x % p ** (agree + 1) for x in diff)
    det3 = berkowitz_charpoly(res[3].C.tolist())[10] % p ** 5
    assert det3 % p ** 3 == 1 and det3 not in (1, p ** 5 - 1)
    N1 = pins.count_points(n, d, p, c, 1)
    assert N1 == 1431
    for N in (3, 4):
        cp = berkowitz_charpoly(res[N].F.tolist())
        a1 = cp[1] % p ** 3
        assert (a1 - p ** 3 if a1 > p ** 3 // 2 else a1) == pins.counts_to_charpoly_prefix(n, p, [N1])[1] == -33
        assert cp[2] % p ** 4 == 605    # a_2 = 605 from #X(F_121) = 1 786 445 (a 16-minute count, not repeated here)


@pytest.mark.skipif(not os.environ.get("ZETA_SLOW_ORACLE"), reason="about 15 minutes; set ZETA_SLOW_ORACLE=1")
def test_cubic_threefold_f11_full_zeta_function():
    """The same cubic threefold at N = 5 (arithmetic mod 11^10): the columns are correct to 4 and 5 digits, one
    short of r = (5, 6), but det C is +-1 and P(T) lifts, to the polynomial that N = 6 (which reaches r; a
    28-minute run) also gives.  Its reciprocal roots all have absolute value 11^(3/2), a_1 and a_2 equal those of
    the point counts (#X(F_11) = 1431, #X(F_121) = 1 786 445), and the first five slopes are 1 (ordinary:
    slope-one length 5)."""
    n, d, p = 4, 3, 11
    att = 0
    while True:
        c = zi.dense_candidate(n, d, p, 11, 0, att)
        att += 1
        if cohomology.is_smooth(n, d, p, c) and cohomology.is_S_smooth(n, d, p, c, (4,)):
            break
    res = zeta.compute_zeta(n, d, p, c, policy="p_chunk", S=(4,), N=5)
    assert res.prec.M == 10
    P = res.P
    assert P[:3] == [1, -33, 605]
    assert pins.count_points(n, d, p, c, 1) == 1431
    assert pins.root_moduli_ok(n, p, P)
    assert pins.newton_above_hodge(n, p, P, [m for m, _ in res.basis])
    from paper_2602_24155_gb300.newton import first_slope_length, newton_slopes
    assert first_slope_length(P, p, 1) == 5 and newton_slopes(P, p) == [1] * 5 + [2] * 5


@pytest.mark.skipif(not os.environ.get("ZETA_SLOW_ORACLE"), reason="about 45 minutes; set ZETA_SLOW_ORACLE=1")
def test_fermat_cubic_threefold_f7_closed_form():
    """x_0^3 + ... + x_4^3 over F_7 (p = 1 mod 3), S = {4}, at the precision rules' N = 10, M = 16: P(T) equals
    Weil's Gauss-sum formula, a closed form computed without any of the reduction."""
    res = zeta.compute_zeta(4, 3, 7, zi.fermat(4, 3), policy="p_chunk", S=(4,))
    assert res.prec.M == 16
    assert res.P == pins.fermat_charpoly(4, 3, 7)
