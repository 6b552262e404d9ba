"""CPU checks of the library's host steps (setup and finish) against the oracle.

The device recurrence is replayed here in plain Python on the plan the
library exports (start terms, section, final map): depth-first chunks with
step matrices generated from the section by the monomial formula
  R_{u,v}[omega, mu] = sum_i (u_i + omega_i) Sec[(i, omega - 1 + e_i), v + mu - 1],
then the library's own finishing step.  Agreement of Y and P(T) with the
oracle checks the host setup, the formula and the finish without a GPU.
"""
import numpy as np
import pytest

import zeta_inputs as zi
from oracle import cohomology, zeta as ozeta
from oracle.algebra import monomials
from oracle.policies import greedy_v, k_max

z = pytest.importorskip("paper_2602_24155_gb300")


def _rank_table(nv, deg):
    return {m: i for i, m in enumerate(monomials(nv, deg))}


def replay(spec, plan):
    n, d, p, coeffs = spec
    nv = n + 1
    q = int(plan["q"])
    b = plan["b"]
    mS = monomials(nv, d * n - n)
    s = len(mS)
    src = _rank_table(nv, n * (d - 2))
    kap = _rank_table(nv, (n + 1) * (d - 2) + 1)
    hpos = _rank_table(nv, d * n - n - 1)
    nsrc = len(src)
    sec = plan["sec"].astype(object)
    H = np.zeros((len(hpos), b), dtype=object)
    for ci in range(plan["U"].shape[0]):
        U = tuple(int(x) for x in plan["U"][ci])
        W = np.zeros((s, b), dtype=object)
        t0, t1 = plan["chain_terms"][ci]
        for t in range(t0, t1):
            r, c = plan["term_rc"][t]
            W[r, c] = (W[r, c] + int(plan["term_coeff"][t])) % q
        while sum(U) > n:
            v = greedy_v(d, U, set(range(nv)))
            k = k_max(U, v, n, d)
            x = tuple(a - k * bb for a, bb in zip(U, v))
            A = np.zeros((s, s), dtype=object)
            B = np.zeros((s, s), dtype=object)
            for j, mu in enumerate(mS):
                g = tuple(v[t] + mu[t] - 1 for t in range(nv))
                if min(g) < 0:
                    continue
                col = kap[g]
                for r, om in enumerate(mS):
                    a = bb = 0
                    for i in range(nv):
                        nu = tuple(om[t] - 1 + (1 if t == i else 0) for t in range(nv))
                        if min(nu) < 0:
                            continue
                        val = sec[i * nsrc + src[nu], col]
                        a += v[i] * val
                        bb += (x[i] + om[i]) * val
                    A[r, j] = a % q
                    B[r, j] = bb % q
            W = ozeta.horner_python(A, B, W, k, q)
            U = x
        for j, mu in enumerate(mS):
            g = tuple(U[t] + mu[t] - 1 for t in range(nv))
            if min(g) < 0:
                continue
            H[hpos[g]] = (H[hpos[g]] + W[j]) % q
    return H.astype(np.uint64)


def test_plan_sizes_match_oracle_precision():
    n, d, p, c, _ = zi.draw_instance("quartic_curve_f11", 0, cohomology.is_smooth)
    b, r, M, s = z.zeta_query((n, d, p, c))
    res = ozeta.compute_zeta(n, d, p, c, want_P=False)
    assert (b, r, M) == (len(res.basis), max(res.prec.r.values()), res.prec.M)
    assert s == 28
    for i in range(1, 4):
        n, d, p, c, _ = zi.draw_instance("quintic_curves", i, cohomology.is_smooth)
        from oracle.precision import Precision
        X = cohomology.Hypersurface(n, d, p, c)
        basis = cohomology.cohomology_basis(X)
        pr = Precision(n, d, p, [m for m, _ in basis])
        assert z.zeta_query((n, d, p, c))[:3] == (len(basis), max(pr.r.values()), pr.M)


def test_replayed_plan_matches_oracle_quartic():
    n, d, p, c, _ = zi.draw_instance("quartic_curve_f11", 0, cohomology.is_smooth)
    spec = (n, d, p, c)
    plan = z.zeta_plan(spec)
    H = replay(spec, plan)
    F, Y, P = z.zeta_finish(spec, H)
    res = ozeta.compute_zeta(n, d, p, c)
    assert (Y.astype(object) == res.Y).all()
    assert P == res.P
    assert (F.astype(object) == res.F).all()


def test_non_smooth_and_unsupported_inputs_are_rejected():
    c = [1 if m in [(4, 0, 0), (0, 4, 0)] else 0 for m in monomials(3, 4)]
    with pytest.raises(z.ZetaError) as e:
        z.zeta_query((2, 4, 7, c))
    assert e.value.status == 2
    with pytest.raises(z.ZetaError) as e:
        z.zeta_query((2, 4, 5, zi.fermat(2, 4)))       # p < 7
    assert e.value.status == 3
    with pytest.raises(z.ZetaError) as e:
        z.zeta_query((2, 4, 11, [11] + [0] * 14))      # coefficient not reduced
    assert e.value.status == 1


@pytest.mark.parametrize("policy", ["depth_first", "p_chunk", "var_by_var"])
@pytest.mark.parametrize("which", [("quartic_curve_f11", 0), ("quintic_curves", 0)])
def test_host_game_matches_the_oracle_game(policy, which):
    # the library's scheduler and the oracle's policies are separate code: same moves, same counts
    n, d, p, c, _ = zi.draw_instance(*which, cohomology.is_smooth)
    plan = z.zeta_plan((n, d, p, c), policy=policy)
    res = ozeta.compute_zeta(n, d, p, c, policy=policy, want_P=False)
    g = plan["game"]
    assert (g["chunks"], g["steps"], g["merges"]) == (res.log.chunks, res.log.steps, res.log.merges)
    assert g["column_steps"] >= res.log.column_steps


def test_cover_policy_plays_fewer_column_steps_with_valid_plans():
    """The cover search (destinations chosen so that terms merge) against p-chunk on the same instances; every
    plan passes the library's legality check (zeta_plan fails otherwise)."""
    import zeta_inputs as zi
    import paper_2602_24155_gb300 as z
    from oracle import cohomology
    tot = {"p_chunk": 0, "cover": 0}
    for i in range(6):
        n, d, p, c, _ = zi.draw_instance("quintic_curves", i, cohomology.is_smooth)
        for pol in tot:
            tot[pol] += z.zeta_plan((n, d, p, c), policy=pol)["game"]["column_steps"]
    assert tot["cover"] < 0.85 * tot["p_chunk"]
    # K3: d = n + 1 leaves no freedom in the destinations, the cover game is the p-chunk game
    n, d, p, c, _ = zi.draw_instance("quartic_k3", 3, cohomology.is_smooth)
    a = z.zeta_plan((n, d, p, c), policy="cover", r=1)["game"]
    b = z.zeta_plan((n, d, p, c), policy="p_chunk", r=1)["game"]
    assert a["column_steps"] == b["column_steps"]


def _step_matrices(spec, plan, U, v, k):
    """A and B of a chunk of k steps from U in direction v (M(y) = yA + B for u = x + y v, x = U - k v), generated
    from the exported section by the monomial formula."""
    n, d, p, coeffs = spec
    nv = n + 1
    q = int(plan["q"])
    mS = monomials(nv, d * n - n)
    s = len(mS)
    src = _rank_table(nv, n * (d - 2))
    kap = _rank_table(nv, (n + 1) * (d - 2) + 1)
    nsrc = len(src)
    sec = plan["sec"]
    x = tuple(a - k * bb for a, bb in zip(U, v))
    A = np.zeros((s, s), dtype=object)
    B = np.zeros((s, s), dtype=object)
    for j, mu in enumerate(mS):
        g = tuple(v[t] + mu[t] - 1 for t in range(nv))
        if min(g) < 0:
            continue
        col = kap[g]
        for r, om in enumerate(mS):
            a = bb = 0
            for i in range(nv):
                nu = tuple(om[t] - 1 + (1 if t == i else 0) for t in range(nv))
                if min(nu) < 0:
                    continue
                val = int(sec[i * nsrc + src[nu], col])
                a += v[i] * val
                bb += (x[i] + om[i]) * val
            A[r, j] = a % q
            B[r, j] = bb % q
    return A, B, x


def _step_matrices_from_tables(spec, plan, tables, U, v, k):
    """A and B as the device forms them from the exported index tables (zeta_plan_tables): with e_j = monoS[j],
    column j reads Sec column rank_kappa(v + e_j - 1), row r reads Sec rows secrow[i][r], weights v_i (A) and
    x_i + e_{r,i} (B).  No knowledge of S is used here: it is all in the tables and the section."""
    n, d, p, coeffs = spec
    nv = n + 1
    q = int(plan["q"])
    e = [tuple(int(a) for a in row) for row in tables["monoS"]]
    secrow = tables["secrow"]
    s = len(e)
    kap = _rank_table(nv, int(plan["kappa"]))
    sec = plan["sec"]
    x = tuple(a - k * bb for a, bb in zip(U, v))
    A = np.zeros((s, s), dtype=object)
    B = np.zeros((s, s), dtype=object)
    for j in range(s):
        g = tuple(v[t] + e[j][t] - 1 for t in range(nv))
        if min(g) < 0:
            continue
        col = kap[g]
        for r in range(s):
            a = bb = 0
            for i in range(nv):
                row = int(secrow[i][r])
                if row < 0:
                    continue
                val = int(sec[row, col])
                a += v[i] * val
                bb += (x[i] + e[r][i]) * val
            A[r, j] = a % q
            B[r, j] = bb % q
    return A, B, x


def replay_moves(spec, plan, moves, tables=None):
    """The device executor's semantics in plain Python: phase by phase, every entry starts from its arrival block
    and/or its start chain, plays its chunks (Algorithm 2), then is stored or added into its destination block of
    the next phase, or accumulated into the numerators at pole order n.  With `tables` the step matrices and the
    numerator exponents come from the device's index tables (any S); without, from the S = {0..n} formula."""
    n, d, p, coeffs = spec
    nv = n + 1
    q = int(plan["q"])
    b = plan["b"]
    mS = monomials(nv, d * n - n) if tables is None else [tuple(int(a) for a in r) for r in tables["monoS"]]
    s = len(mS)
    hpos = _rank_table(nv, d * n - n - 1)
    base = n if tables is None else len(plan["S"]) - 1
    H = np.zeros((len(hpos), b), dtype=object)
    ph, ent, chk = moves["phase_begin"], moves["entries"], moves["chunks"]
    cur = {}
    cache = {}
    for f in range(len(ph) - 1):
        nxt = {}
        for ei in range(int(ph[f]), int(ph[f + 1])):
            row = [int(x) for x in ent[ei]]
            U = tuple(row[:nv])
            c0, c1, arrival, start, dest, flags, live = row[nv:nv + 7]
            W = cur[arrival].copy() if arrival >= 0 else np.zeros((s, b), dtype=object)
            if start >= 0:
                t0, t1 = plan["chain_terms"][start]
                for t in range(int(t0), int(t1)):
                    r, c = plan["term_rc"][t]
                    W[r, c] = (W[r, c] + int(plan["term_coeff"][t])) % q
            for ci in range(c0, c1):
                v = tuple(int(x) for x in chk[ci][:nv])
                k = int(chk[ci][nv])
                key = (U, v, k)
                if key not in cache:
                    cache[key] = (_step_matrices(spec, plan, U, v, k) if tables is None
                                  else _step_matrices_from_tables(spec, plan, tables, U, v, k))
                A, B, x = cache[key]
                W = ozeta.horner_python(A, B, W, k, q)
                U = x
            assert all((live >> c) & 1 or not W[:, c].any() for c in range(b))
            if dest < 0:
                assert sum(U) == base
                for j, mu in enumerate(mS):
                    g = tuple(U[t] + mu[t] - 1 for t in range(nv))
                    if min(g) < 0:
                        continue
                    H[hpos[g]] = (H[hpos[g]] + W[j]) % q
            elif flags & 1:
                nxt[dest] = W
            else:
                nxt[dest] = (nxt[dest] + W) % q
        cur = nxt
    return H.astype(np.uint64)


@pytest.mark.parametrize("policy", ["p_chunk", "cover", "var_by_var", "learned"])
def test_replayed_moves_of_every_policy_match_oracle(policy):
    """The exact moves the device would execute (zeta_plan_moves), replayed with exact arithmetic: Y, F and P(T)
    equal the oracle's for the paper's policies, the cover search and the learned policy (a network with random
    weights still yields a legal plan)."""
    n, d, p, c, _ = zi.draw_instance("quartic_curve_f11", 0, cohomology.is_smooth)
    spec = (n, d, p, c)
    opt = {"policy": policy}
    if policy == "learned":
        opt.update(weights=z.zeta_mlp_init(8, 3), hidden=8)
    plan = z.zeta_plan(spec, **opt)
    moves = z.zeta_plan_moves(spec, **opt)
    assert len(moves["entries"]) == plan["game"]["entries"]
    H = replay_moves(spec, plan, moves)
    F, Y, P = z.zeta_finish(spec, H)
    res = ozeta.compute_zeta(n, d, p, c)
    assert (Y.astype(object) == res.Y).all()
    assert P == res.P


@pytest.mark.parametrize("policy", ["cover", "learned"])
def test_replayed_moves_on_a_quintic_at_precision_one(policy):
    # a non-ordinary plane quintic over F_7 at relative precision 1 (P mod p): the cover levels have freedom d - 3 = 2
    n, d, p, c, _ = zi.draw_instance("quintic_curves", 12, cohomology.is_smooth)
    spec = (n, d, p, c)
    opt = {"policy": policy, "r": 1}
    if policy == "learned":
        opt.update(weights=z.zeta_mlp_init(8, 5), hidden=8)
    plan = z.zeta_plan(spec, **opt)
    moves = z.zeta_plan_moves(spec, **opt)
    H = replay_moves(spec, plan, moves)
    F, Y, P = z.zeta_finish(spec, H, r=1)
    res = ozeta.compute_zeta(n, d, p, c, r=1)
    assert (Y.astype(object) == res.Y).all()
    assert [a % p for a in P] == [a % p for a in res.P]


def test_moduli_above_2_60_are_rejected():
    """The device keeps residues as two 30-bit limbs (and at most eight balanced base-256 digits on the tensor
    cores): a plane quintic over F_37 at relative precision 6 needs p^M = 37^12 = 2^62.5 and is refused before any
    device work, while its default precision (below 2^60) is accepted."""
    import zeta_inputs as zi
    from oracle import cohomology
    n, d, p, c, _ = zi.draw_instance("quintic_curves", 8, cohomology.is_smooth)
    assert p == 37
    b, r, M, s = z.zeta_query((n, d, p, c))
    assert p ** M < 2 ** 60
    with pytest.raises(z.ZetaError) as err:
        z.zeta_query((n, d, p, c), r=6)
    assert err.value.status == 4


# ---------------------------------------------------------------------------
# General S (Prop. 3.3 with S other than {0..n}): the same device tables and kernel formula
# ---------------------------------------------------------------------------
def _cubic_surface(p, seed=7):
    att = 0
    while True:
        c = zi.dense_candidate(3, 3, p, seed, p, att)
        att += 1
        if cohomology.is_smooth(3, 3, p, c) and cohomology.is_S_smooth(3, 3, p, c, (3,)):
            return (3, 3, p, c)


@pytest.mark.parametrize("which", [("quartic_curve_f11", 0), ("quintic_curves", 3)])
def test_device_tables_for_S_all_are_the_monomial_formula(which):
    n, d, p, c, _ = zi.draw_instance(*which, cohomology.is_smooth)
    nv = n + 1
    tab = z.zeta_plan_tables((n, d, p, c))
    mS = monomials(nv, d * n - n)
    assert [tuple(r) for r in tab["monoS"]] == mS
    src = _rank_table(nv, n * (d - 2))
    for i in range(nv):
        for r, om in enumerate(mS):
            nu = tuple(om[t] - 1 + (1 if t == i else 0) for t in range(nv))
            assert tab["secrow"][i][r] == (-1 if min(nu) < 0 else i * len(src) + src[nu])


@pytest.mark.parametrize("policy", ["depth_first", "p_chunk", "var_by_var", "cover"])
def test_general_S_replay_on_a_curve_matches_oracle(policy):
    """The quartic over F_11 with S = {1, 2}: the library's section of J_S, start terms, tables and moves, replayed
    through the device formula, give the oracle's Y (which does not depend on S) and P(T)."""
    n, d, p, c, _ = zi.draw_instance("quartic_curve_f11", 0, cohomology.is_smooth)
    spec = (n, d, p, c)
    opt = {"policy": policy, "S": (1, 2)}
    plan = z.zeta_plan(spec, **opt)
    assert plan["S"] == (1, 2) and plan["kappa"] == 3 * 3 + 1 - 2
    H = replay_moves(spec, plan, z.zeta_plan_moves(spec, **opt), z.zeta_plan_tables(spec, **opt))
    F, Y, P = z.zeta_finish(spec, H, **opt)
    res = ozeta.compute_zeta(n, d, p, c)
    assert (Y.astype(object) == res.Y).all()
    assert P == res.P


@pytest.mark.parametrize("p,policy", [(7, "depth_first"), (7, "p_chunk"), (7, "var_by_var"), (11, "p_chunk")])
def test_general_S_replay_on_cubic_surfaces_matches_oracle(p, policy):
    """Cubic surfaces (d = 3 < n + 1): the library picks S = {3}; its game counts equal the oracle's (separate
    code), and the replayed device formula gives the oracle's Y and P(T)."""
    spec = _cubic_surface(p)
    plan = z.zeta_plan(spec, policy=policy)
    assert plan["S"] == (3,)
    res = ozeta.compute_zeta(*spec, policy=policy, S=(3,))
    g = plan["game"]
    assert (g["chunks"], g["steps"], g["merges"]) == (res.log.chunks, res.log.steps, res.log.merges)
    H = replay_moves(spec, plan, z.zeta_plan_moves(spec, policy=policy), z.zeta_plan_tables(spec, policy=policy))
    F, Y, P = z.zeta_finish(spec, H)
    assert (Y.astype(object) == res.Y).all()
    assert P == res.P


def test_cover_on_cubic_surfaces_replays_exactly_and_saves_steps():
    """The cover search with S = {3}: boxes U - L 1_S (only x_3 must fall every step), paths taking d - |S| = 2 free
    units per step.  The replayed plan gives the oracle's Y and P(T); over 12 surfaces it plays far fewer column
    steps than p-chunk."""
    spec = _cubic_surface(7)
    plan = z.zeta_plan(spec, policy="cover")
    H = replay_moves(spec, plan, z.zeta_plan_moves(spec, policy="cover"), z.zeta_plan_tables(spec, policy="cover"))
    F, Y, P = z.zeta_finish(spec, H)
    res = ozeta.compute_zeta(*spec, policy="p_chunk", S=(3,))
    assert (Y.astype(object) == res.Y).all()
    assert P == res.P
    tot = {"p_chunk": 0, "cover": 0}
    for i in range(12):
        n, d, p, c, _ = zi.draw_instance("cubic_surfaces", i, lambda *a: cohomology.is_smooth(*a)
                                         and cohomology.is_S_smooth(*a, (3,)))
        for pol in tot:
            tot[pol] += z.zeta_plan((n, d, p, c), policy=pol)["game"]["column_steps"]
    assert tot["cover"] < 0.7 * tot["p_chunk"]


def test_general_S_refusals():
    n, d, p, c, _ = zi.draw_instance("quartic_curve_f11", 0, cohomology.is_smooth)
    with pytest.raises(z.ZetaError) as e:
        z.zeta_query((n, d, p, c), S=(2,))            # not {2}-smooth (oracle: is_S_smooth is False)
    assert e.value.status == 2 and not cohomology.is_S_smooth(n, d, p, c, (2,))
    with pytest.raises(z.ZetaError) as e:
        z.zeta_query((n, d, p, c), S=(3,))            # x_3 does not exist in P^2
    assert e.value.status == 1
    with pytest.raises(z.ZetaError) as e:
        z.zeta_plan((n, d, p, c), policy="learned", S=(1, 2))
    assert e.value.status == 3
    spec = _cubic_surface(7)
    with pytest.raises(z.ZetaError) as e:
        z.zeta_query(spec, S=(0, 1, 2, 3))            # |S| = 4 > d = 3
    assert e.value.status == 3
    fermat4 = (5, 3, 7, zi.fermat(5, 3))               # cubic fourfold: s = C(15, 5) = 3003
    with pytest.raises(z.ZetaError) as e:
        z.zeta_query(fermat4)                          # full precision: p^M = 7^25 > 2^60
    assert e.value.status == 4
    assert z.zeta_query(fermat4, r=1) == (22, 1, 9, 3003)   # b, r, M, s at relative precision 1
    with pytest.raises(z.ZetaError) as e:
        z.zeta_plan(fermat4, r=1)                      # s > 512: the right inverses are solved on the device only
    assert e.value.status == 3


def test_cubic_threefold_is_planned_with_S_n():
    """A cubic threefold over F_11 (n = 4, d = 3, s = 495): S = {4}, kappa = 10, and the precision rules give
    r = 6, M = 16; the host plans it (a legal plan, checked move by move), the device is not run here."""
    n, d, p = 4, 3, 11
    att = 0
    while True:
        c = zi.dense_candidate(n, d, p, 11, 0, att)
        att += 1
        try:
            b, r, M, s = z.zeta_query((n, d, p, c))
            break
        except z.ZetaError as e:
            assert e.status == 2
    assert (b, r, M, s) == (10, 6, 16, 495)
    assert cohomology.is_S_smooth(n, d, p, c, (4,))          # the oracle's test accepts the same instance
    plan = z.zeta_plan((n, d, p, c), policy="p_chunk")
    assert plan["S"] == (4,) and plan["kappa"] == 10
    assert plan["game"]["column_steps"] > 0


def _oracle_game_counts(n, d, p, c, policy, S, r):
    """The oracle's policy played on exponents only (no matrices): start terms of Prop. 2.1 after Tweak, combined
    by u, then oracle.policies.play; returns (chunks, steps, merges)."""
    from oracle.policies import play, GameLog
    from oracle.precision import Precision
    X = cohomology.Hypersurface(n, d, p, c)
    basis = cohomology.cohomology_basis(X)
    prec = Precision(n, d, p, [m for m, _ in basis], r=r)
    us = []
    seen = set()
    for col, U, J, val in ozeta.frobenius_terms(X, basis, prec, S):
        if U not in seen:
            seen.add(U)
            us.append(U)
    log = GameLog()

    def reduce_chunk(u, v, k, w):
        log.chunks += 1
        log.steps += k
        return w
    play(policy, [(u, None) for u in us], n, d, p, S, reduce_chunk, lambda a, b: a, log)
    return log.chunks, log.steps, log.merges


@pytest.mark.parametrize("case,policy", [("k3_S3", "depth_first"), ("k3_S3", "p_chunk"), ("k3_S3", "var_by_var"),
                                         ("threefold_S4", "p_chunk")])
def test_host_game_with_S_n_matches_the_oracle_game(case, policy):
    # K3 surfaces admit both S = {0..3} and S = {3}; cubic threefolds only S = {4}.  At relative precision 1 the
    # library's scheduler and the oracle's policies (separate code) play the same moves.
    if case == "k3_S3":
        n, d, p, c, _ = zi.draw_instance("quartic_k3", 1, cohomology.is_smooth)
        S = (3,)
        if not cohomology.is_S_smooth(n, d, p, c, S):
            pytest.skip("instance not {3}-smooth")
    else:
        n, d, p, S = 4, 3, 11, (4,)
        att = 0
        while True:
            c = zi.dense_candidate(n, d, p, 11, 0, att)
            att += 1
            try:
                z.zeta_query((n, d, p, c))
                break
            except z.ZetaError as e:
                assert e.status == 2
    g = z.zeta_plan((n, d, p, c), policy=policy, r=1, S=S)["game"]
    assert (g["chunks"], g["steps"], g["merges"]) == _oracle_game_counts(n, d, p, c, policy, S, 1)


def test_quintic_surface_plans_with_52_columns():
    """Quintic surfaces (b = 52 > 32): the host plans them with 64-bit column masks (relative precision 1, M = 3);
    every term's columns are carried, and zeta_plan_moves, whose `live` export is one 32-bit word, refuses them."""
    spec = (3, 5, 7, zi.fermat(3, 5))
    P = z.zeta_plan(spec, r=1, policy="p_chunk")
    assert P["b"] == 52 and P["s"] == 455 and P["M"] == 3
    g = P["game"]
    assert g["chunks"] > 0 and g["column_steps"] >= g["steps"]
    assert set(int(c) for c in P["term_rc"][:, 1]) <= set(range(52))
    assert max(int(c) for c in P["term_rc"][:, 1]) >= 32
    with pytest.raises(z.ZetaError) as e:
        z.zeta_plan_moves(spec, r=1, policy="p_chunk")
    assert e.value.status == 3


def test_plan_sizes_match_the_setup():
    """The output sizes the device-setup binding allocates without running the setup equal zeta_plan's: plane
    quartics and quintics, a cubic surface (S = {3}), a quartic K3 and S chosen by the caller."""
    cases = [((2, 4, 11, zi.draw_instance("quartic_curve_f11", 0, cohomology.is_smooth)[3]), {}),
             ((2, 5, 13, zi.draw_instance("quintic_curves", 2, cohomology.is_smooth)[3]), {}),
             ((3, 3, 7, _cubic_surface(7)[3]), {}),
             ((3, 4, 7, zi.fermat(3, 4)), {}),
             ((2, 4, 11, zi.draw_instance("quartic_curve_f11", 0, cohomology.is_smooth)[3]), {"S": (1, 2)})]
    for spec, opt in cases:
        P = z.zeta_plan(spec, policy="p_chunk", **opt)
        assert z.plan_sizes(spec, **opt) == (P["b"], P["sec"].shape[0], P["sec"].shape[1], P["fin"].shape[1])
