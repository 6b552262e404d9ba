"""The stored P(T) of the dense cubic threefold over F_11 (tests/golden/cubic_threefold_f11.txt, written by
tests/golden/make_golden.py threefold from the oracle alone) against what fixes it independently: the instance is
the recipe's own draw, #X(F_11) from a brute-force count (a_1), every reciprocal root has absolute value 11^(3/2),
and the Newton polygon lies on or above the Hodge polygon (slopes 1 and 2, five each)."""
import os

import zeta_inputs as zi
from oracle import cohomology, pins

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


def test_golden_threefold_is_the_recipes_draw():
    n, d, p, c, P = _golden()
    att = 0
    while True:
        cand = zi.dense_candidate(n, d, p, 11, 0, att)
        att += 1
        if cohomology.is_smooth(n, d, p, cand) and cohomology.is_S_smooth(n, d, p, cand, (4,)):
            break
    assert cand == c and len(P) == 11 and P[0] == 1


def test_golden_threefold_counts_and_weil():
    n, d, p, c, P = _golden()
    assert pins.charpoly_to_counts(n, p, P, 1) == [pins.count_points(n, d, p, c, 1)] == [1431]
    assert pins.root_moduli_ok(n, p, P)
    assert pins.newton_above_hodge(n, p, P, [2] * 5 + [3] * 5)
