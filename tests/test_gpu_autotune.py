"""The batch engine's autotuner, the automatic path and the block-size option (GPU)."""
import pytest

import zeta_inputs as zi
from oracle import cohomology, zeta as ozeta

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


def _instance(workload, i):
    n, d, p, c, _ = zi.draw_instance(workload, i, cohomology.is_smooth)
    return n, d, p, c


def test_autotune_times_every_candidate_and_auto_uses_the_choice(ctx):
    specs = [_instance("quintic_curves", i) for i in range(96)]
    t = z.zeta_autotune(ctx, specs, sample=48, policy="p_chunk")
    assert t["n"] == 2 and t["d"] == 5 and t["sample"] == 48
    paths = [c["path"] for c in t["candidates"]]
    assert paths.count("vector") == 4 and paths.count("gemm") == 1
    assert all(c["ms"] > 0 for c in t["candidates"])
    assert t["best"]["ms"] == min(c["ms"] for c in t["candidates"])
    # the default sample is 16 instances per SM, capped by the batch
    assert z.zeta_autotune(ctx, specs[:40], policy="p_chunk")["sample"] == 40
    out_auto, _, _ = z.zeta_batch(ctx, specs[:24], policy="p_chunk", path="auto")
    out_vec, _, _ = z.zeta_batch(ctx, specs[:24], policy="p_chunk", path="vector")
    assert out_auto == out_vec
    ref = ozeta.compute_zeta(*specs[0])
    assert out_auto[0] == ref.P


def test_auto_without_tuning_falls_back_to_the_vector_path(ctx):
    n, d, p, c = _instance("quartic_curve_f11", 0)   # (2, 4) is never tuned in this module
    P_auto, _ = z.zeta_charpoly(ctx, (n, d, p, c), path="auto")
    P_vec, _ = z.zeta_charpoly(ctx, (n, d, p, c), path="vector")
    assert P_auto == P_vec == ozeta.compute_zeta(n, d, p, c).P


@pytest.mark.parametrize("threads", [64, 96, 256, 512])
def test_block_threads_option_keeps_results(ctx, threads):
    spec = _instance("quintic_curves", 5)
    P, _ = z.zeta_charpoly(ctx, spec, policy="p_chunk", block_threads=threads)
    P0, _ = z.zeta_charpoly(ctx, spec, policy="p_chunk")
    assert P == P0


def test_bad_block_threads_and_mixed_classes_are_rejected(ctx):
    spec = _instance("quintic_curves", 5)
    with pytest.raises(z.ZetaError):
        z.zeta_charpoly(ctx, spec, block_threads=100)
    with pytest.raises(z.ZetaError):
        z.zeta_autotune(ctx, [spec, _instance("quartic_curve_f11", 0)])


def test_bounded_wait_gives_up_and_the_context_stays_usable(ctx):
    # failure detection without a GPU fault: a wait on a barrier nothing arrives on runs out after its limit
    st, waited = z.zeta_selftest_wait(ctx, 200)
    assert st == 6 and 200.0 <= waited < 5000.0
    spec = _instance("quartic_curve_f11", 0)
    P, _ = z.zeta_charpoly(ctx, spec, path="gemm")
    assert P == ozeta.compute_zeta(*spec).P
