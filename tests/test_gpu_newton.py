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


def test_k3_heights_from_a_precision_one_batch(ctx):
    """Quartic K3 surfaces (s = 220, b = 21) in one launch at relative precision 1: heights checked against the
    Hasse-Witt matrix (a_1 mod p, an independent computation), the Fermat surfaces (supersingular for p = 3 mod 4)
    and the oracle's own precision-1 run."""
    import zeta_inputs as zi
    from oracle import cohomology, pins, zeta as ozeta
    from paper_2602_24155_gb300.newton import k3_heights
    idx = list(range(8)) + [12, 24]
    specs = [zi.draw_instance("quartic_k3", i, cohomology.is_smooth)[:4] for i in idx]
    specs += [(3, 4, 7, zi.fermat(3, 4)), (3, 4, 13, zi.fermat(3, 4))]
    heights, per, tot = k3_heights(ctx, specs)
    assert tot["kernel_launches"] == 1 and all(h is not None for h in heights)
    assert heights[-2] == "inf" and heights[-1] == 1
    for (n, d, p, c), h in zip(specs[:-2], heights[:-2]):
        a1 = pins.hasse_witt_charpoly_mod_p(n, d, p, c)[1] % p
        assert (h == 1) == (a1 != 0)
    P_gpu = z.zeta_charpoly(ctx, specs[8], policy="p_chunk", r=1)[0]
    assert P_gpu == ozeta.compute_zeta(*specs[8], r=1).P
