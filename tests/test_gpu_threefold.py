"""Cubic threefolds (n = 4, d = 3: s = 495, b = 10, S = {4}) on the cluster executor at full precision.

d < n + 1, so the reduction runs with the index set S = {4} of Prop. 3.3; the
step matrices (495 x 495, mod 11^16 or 7^16) are spread over a cluster of CTAs.
 - The Fermat cubic threefold over F_7 (p = 1 mod 3) against Weil's Gauss-sum
   formula (a closed form computed without any of the reduction).
 - A dense cubic threefold over F_11 against the oracle's P(T), stored in
   tests/golden/cubic_threefold_f11.txt (written by make_golden.py threefold
   from the oracle alone), and against #X(F_11) and the Weil bounds.
"""
import os

import pytest

import zeta_inputs as zi
from oracle import cohomology, pins

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
z = pytest.importorskip("paper_2602_24155_gb300")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cubic_threefold_f11.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or ":" not in line:
            continue
        key, _, val = line.partition(":")
        out[key.strip()] = val.strip()
    n, d, p = map(int, out["n d p"].split())
    return n, d, p, [int(x) for x in out["coeffs"].split()], [int(x) for x in out["P"].split()]


@pytest.fixture(scope="module")
def threefolds():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    ctx = z.zeta_create(0, torch.cuda.current_stream().cuda_stream)
    n, d, p, c, P_ref = _golden()
    specs = [(4, 3, 7, zi.fermat(4, 3)), (n, d, p, c)]
    P, per, tot = z.zeta_batch(ctx, specs, policy="p_chunk")
    z.zeta_destroy(ctx)
    return specs, P, per, P_ref


def test_fermat_cubic_threefold_f7(threefolds):
    specs, P, per, _ = threefolds
    assert per[0]["status"] == 0 and per[0]["s"] == 495
    assert P[0] == pins.fermat_charpoly(4, 3, 7)


def test_dense_cubic_threefold_f11_equals_the_oracle(threefolds):
    specs, P, per, P_ref = threefolds
    n, d, p, c = specs[1]
    assert per[1]["status"] == 0
    assert P[1] == P_ref
    assert pins.charpoly_to_counts(n, p, P[1], 1) == [pins.count_points(n, d, p, c, 1)]
    assert pins.root_moduli_ok(n, p, P[1])


def test_newton_strata_search_over_cubic_threefolds():
    """The paper's Method 1 (Sec. 5.1) over cubic threefolds: random dense cubics over F_11, the slope-one length
    (the p-rank analogue of Sec. 1.2) from a relative-precision-1 batch, then full precision for the non-ordinary
    ones (length <= 4), whose P(T) must satisfy #X(F_11), Weil and the filter's own count."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2602_24155_gb300.newton import first_slope_length, search
    ctx = z.zeta_create(0, torch.cuda.current_stream().cuda_stream)
    try:
        out = search(ctx, 4, 3, 11, 80, seed=2)
    finally:
        z.zeta_destroy(ctx)
    print("cubic threefolds over F_11:", {k: v for k, v in out.items() if k != "strata"},
          {lab: len(v) for lab, v in out["strata"].items()})
    assert out["smooth"] >= 8          # about one in six random cubics is smooth and {4}-smooth over F_11
    assert sum(out["p_rank"].values()) == out["smooth"]
    assert set(out["p_rank"]) <= set(range(6))
    assert out["kept"] == sum(len(v) for v in out["strata"].values())
    for items in out["strata"].values():
        for coeffs, P in items:
            assert len(P) == 11 and P[0] == 1
            assert pins.root_moduli_ok(4, 11, P)
            assert pins.charpoly_to_counts(4, 11, P, 1) == [pins.count_points(4, 3, 11, coeffs, 1)]
            assert first_slope_length(P, 11, 1) <= 4
