"""Newton-strata search over the batch engine (GPU): the p-rank filter against full-precision runs."""
import pytest

from paper_2602_24155_gb300.newton import newton_slopes, random_hypersurfaces, search, unit_roots_mod_p

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


def test_filter_run_agrees_with_full_precision(ctx):
    specs = random_hypersurfaces(2, 5, 7, 40, seed=3)
    low, per, _ = z.zeta_batch(ctx, specs, policy="p_chunk", r=1)
    full, per_full, _ = z.zeta_batch(ctx, specs, policy="p_chunk")
    checked = 0
    for P_low, P, st in zip(low, full, per):
        if st["status"] != 0:
            continue
        assert [a % 7 for a in P_low] == [a % 7 for a in P]
        assert unit_roots_mod_p(P_low, 7) == newton_slopes(P, 7).count(0)
        checked += 1
    assert checked >= 30


def test_method_1_search_finds_non_ordinary_curves(ctx):
    out = search(ctx, 2, 5, 7, 300, seed=11)
    assert out["smooth"] > 250
    assert sum(out["p_rank"].values()) == out["smooth"]
    # codimension one: roughly 1/p of the curves are non-ordinary
    assert 10 <= out["kept"] <= 100
    for label, found in out["strata"].items():
        for coeffs, P in found:
            slopes = newton_slopes(P, 7)
            assert slopes.count(0) <= 5 and len(slopes) == 12
            assert slopes == sorted(1 - x for x in slopes)   # symmetric (functional equation)
