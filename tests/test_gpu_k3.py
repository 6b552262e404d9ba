"""Quartic K3 surfaces (n = 3, d = 4: s = 220, b = 21) on the cluster executor.

Instances with s > 128 are reduced by thread-block clusters (each CTA holds a
row slice of the step matrices; the new W rows travel through distributed
shared memory).  These tests pin that path:
 - the unnormalised columns Y equal the oracle's bit for bit at truncated
   series orders (dense and sparse surfaces, p = 7, 11, 13), and at a modulus
   above 2^56, which takes the 20 x 30-bit limb split instead of 28 x 28;
 - at the full precision of the library's rules (r_m, N_m), P(T) of the
   Fermat quartic over F_13 equals Weil's Gauss-sum formula, and P(T) of
   random dense and sparse surfaces agrees with brute-force point counts over
   F_p and F_{p^2}, has every reciprocal root of absolute value p, lies on or
   above the Hodge polygon, and does not change when every N_m grows by one.
"""
import os
import sys

import pytest

import zeta_inputs as zi
from oracle import cohomology, pins, precision, zeta as ozeta

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import k3_golden  # noqa: E402

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


def _k3(i):
    n, d, p, c, _ = zi.draw_instance("quartic_k3", i, cohomology.is_smooth)
    return n, d, p, c


# instance 9 is sparse (7 monomials, p = 7); 1: dense over F_11; 2: dense over F_13
@pytest.mark.parametrize("i", [9, 1, 2])
def test_k3_truncated_columns_on_clusters(ctx, i):
    n, d, p, c = _k3(i)
    N = {1: 2, 2: 1, 3: 1}
    ref = ozeta.compute_zeta(n, d, p, c, N=N, r=2, normalise=False)
    F, Y, st = z.zeta_frobenius(ctx, (n, d, p, c), N=N, r=2, y_only=True, policy="p_chunk")
    assert st["s"] == 220 and st["b"] == 21
    assert (Y.astype(object) == ref.Y).all()


def test_k3_columns_with_a_modulus_above_2_56(ctx):
    # r = 20 at N = 1: q = 7^20 = 2^56.15 takes the 20 x 30-bit limb split of the cluster executor
    n, d, p, c = _k3(0)
    b, r, M, s = z.zeta_query((n, d, p, c), r=20, N=1)
    assert p ** M >= 1 << 56
    ref = ozeta.compute_zeta(n, d, p, c, N=1, r=20, normalise=False)
    F, Y, st = z.zeta_frobenius(ctx, (n, d, p, c), N=1, r=20, y_only=True, policy="depth_first")
    assert (Y.astype(object) == ref.Y).all()


FULL = [("fermat", 13), ("k3", 0), ("k3", 9), ("k3", 1), ("k3", 2)]   # p = 13, 7 (dense), 7 (sparse), 11, 13


@pytest.fixture(scope="module")
def full_precision(ctx):
    """Full-precision P(T) of the FULL instances in one batch (one persistent launch)."""
    specs = []
    for kind, x in FULL:
        specs.append((3, 4, x, zi.fermat(3, 4)) if kind == "fermat" else _k3(x))
    P, per, tot = z.zeta_batch(ctx, specs, policy="p_chunk")
    assert all(st["status"] == 0 for st in per), per
    return specs, P, per


def test_fermat_k3_over_f13_full_precision(full_precision):
    specs, P, _ = full_precision
    assert P[0] == pins.fermat_charpoly(3, 4, 13)


@pytest.mark.parametrize("idx", [1, 2, 3, 4])
def test_k3_full_precision_counts_and_weil(full_precision, idx):
    specs, P, per = full_precision
    n, d, p, c = specs[idx]
    Pi = P[idx]
    assert len(Pi) == 22 and Pi[0] == 1
    R = 2 if p <= 11 else 1
    counts = [pins.count_points(n, d, p, c, r) for r in range(1, R + 1)]
    assert pins.charpoly_to_counts(n, p, Pi, R) == counts
    assert pins.root_moduli_ok(n, p, Pi)
    X = cohomology.Hypersurface(n, d, p, c)
    pole = [m for m, _ in cohomology.cohomology_basis(X)]
    assert pins.newton_above_hodge(n, p, Pi, pole)


def test_k3_precision_rule_is_stable_under_one_more_term(ctx, full_precision):
    specs, P, per = full_precision
    n, d, p, c = specs[4]
    N = list(per[4]["N"][:n])
    P1, per1, _ = z.zeta_batch(ctx, [specs[4]], policy="p_chunk", N={m + 1: N[m] + 1 for m in range(n)})
    assert per1[0]["status"] == 0
    assert P1[0] == P[4]


def test_k3_full_precision_equals_the_oracle(full_precision):
    specs, P, _ = full_precision
    by_instance = {x: P[i] for i, (kind, x) in enumerate(FULL) if kind == "k3"}
    for g in k3_golden.load():
        assert by_instance[g["instance"]] == g["P"], g["instance"]
