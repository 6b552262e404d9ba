"""The stored full-precision P(T) of three quartic K3 surfaces (tests/golden/quartic_k3_full.txt, written by
tests/golden/make_golden.py k3 from the oracle alone) against what fixes them independently of the oracle:
the instances are the workload's own draws, #X(F_p) (and #X(F_49) at p = 7) from brute-force counts, every
reciprocal root of absolute value p, and the Newton polygon on or above the Hodge polygon (Sec. 2.1, 2.5)."""
import os
import sys

import pytest

import zeta_inputs as zi
from oracle import cohomology, pins

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import k3_golden  # noqa: E402

GOLDEN = k3_golden.load()


def test_golden_file_holds_the_three_surfaces():
    assert [g["instance"] for g in GOLDEN] == [9, 2, 0]
    for g in GOLDEN:
        n, d, p, c, _ = zi.draw_instance("quartic_k3", g["instance"], cohomology.is_smooth)
        assert (n, d, p, c) == (g["n"], g["d"], g["p"], g["coeffs"])
        assert len(g["P"]) == 22 and g["P"][0] == 1


@pytest.mark.parametrize("k", range(3))
def test_golden_k3_counts_and_weil(k):
    g = GOLDEN[k]
    n, d, p, c, P = g["n"], g["d"], g["p"], g["coeffs"], g["P"]
    R = 2 if p == 7 else 1
    assert pins.charpoly_to_counts(n, p, P, R) == [pins.count_points(n, d, p, c, r) for r in range(1, R + 1)]
    assert pins.root_moduli_ok(n, p, P)
    X = cohomology.Hypersurface(n, d, p, c)
    assert pins.newton_above_hodge(n, p, P, [m for m, _ in cohomology.cohomology_basis(X)])
