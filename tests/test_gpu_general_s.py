"""GPU parity of controlled reduction with an index set S other than {0..n} (Prop. 3.3, Definition 3.1).

The kernel is the one of S = {0..n}; what changes is the host's section (of J_S) and the index tables it reads.
Checked against the oracle's general-S computation, the S-independent columns Y of a curve, point counts and
Weil's theorems.
"""
import pytest

import zeta_inputs as zi
from oracle import cohomology, pins, zeta as ozeta

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
z = pytest.importorskip("paper_2602_24155_gb300")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = z.zeta_create(0, torch.cuda.current_stream().cuda_stream)
    yield c
    z.zeta_destroy(c)


def _cubic_surfaces(p, count, seed=21):
    out = []
    att = 0
    while len(out) < count:
        c = zi.dense_candidate(3, 3, p, seed, p, att)
        att += 1
        if cohomology.is_smooth(3, 3, p, c) and cohomology.is_S_smooth(3, 3, p, c, (3,)):
            out.append((3, 3, p, c))
    return out


@pytest.mark.parametrize("policy", ["depth_first", "p_chunk", "var_by_var"])
def test_curve_with_smaller_S_matches_oracle(ctx, policy):
    # the quartic over F_11 with S = {1, 2}: Y is the same as with S = {0..n}
    n, d, p, c, _ = zi.draw_instance("quartic_curve_f11", 0, cohomology.is_smooth)
    ref = ozeta.compute_zeta(n, d, p, c)
    F, Y, _ = z.zeta_frobenius(ctx, (n, d, p, c), policy=policy, S=(1, 2))
    assert (Y.astype(object) == ref.Y).all()
    P, _ = z.zeta_charpoly(ctx, (n, d, p, c), policy=policy, S=(1, 2))
    assert P == ref.P


@pytest.mark.parametrize("policy", ["depth_first", "p_chunk", "var_by_var", "cover"])
def test_cubic_surface_matches_oracle(ctx, policy):
    spec = _cubic_surfaces(7, 1, seed=7)[0]
    ref = ozeta.compute_zeta(*spec, policy="p_chunk", S=(3,))     # Y does not depend on the policy
    F, Y, _ = z.zeta_frobenius(ctx, spec, policy=policy)
    assert (Y.astype(object) == ref.Y).all()
    P, _ = z.zeta_charpoly(ctx, spec, policy=policy)
    assert P == ref.P


@pytest.mark.parametrize("p", [7, 13])
def test_fermat_cubic_surface_closed_form(ctx, p):
    P, _ = z.zeta_charpoly(ctx, (3, 3, p, zi.fermat(3, 3)), policy="p_chunk")
    assert P == pins.fermat_charpoly(3, 3, p)


def test_cubic_surface_batch(ctx):
    # one persistent launch over 48 cubic surfaces (p = 7, 11, 13) mixed with plane quintics (S = {0..n}):
    # every P(T) checked by #X(F_p), Weil, and the first of each prime by the oracle
    specs = []
    for p in (7, 11, 13):
        specs += _cubic_surfaces(p, 16)
    quintics = [zi.draw_instance("quintic_curves", i, cohomology.is_smooth)[:4] for i in range(8)]
    out, per, _ = z.zeta_batch(ctx, specs + quintics, policy="p_chunk")
    assert all(x["status"] == 0 for x in per)
    out_cover, per_cover, _ = z.zeta_batch(ctx, specs + quintics, policy="cover")
    assert all(x["status"] == 0 for x in per_cover)
    assert out_cover == out
    for spec, P in zip(specs, out):
        n, d, p, c = spec
        N1 = pins.count_points(n, d, p, c, 1)
        assert P[:2] == pins.counts_to_charpoly_prefix(n, p, [N1])
        assert pins.root_moduli_ok(n, p, P)
    for k in (0, 16, 32):
        assert out[k] == ozeta.compute_zeta(*specs[k], policy="p_chunk", S=(3,)).P
    for spec, P in zip(quintics[:2], out[len(specs):]):
        assert P == ozeta.compute_zeta(*spec, policy="p_chunk").P
