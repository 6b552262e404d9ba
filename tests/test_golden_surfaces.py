"""The stored Frobenius columns of two quintic surfaces over F_7 at relative precision 1
(tests/golden/quintic_surfaces_r1.txt, written by make_golden.py surface from the oracle).  Checked here on the CPU:
the coefficients are the stated draws, the modulus is p^M = 7^3 of the precision rule at r = 1, and Y has b = 52
rows and columns of residues."""
import os

import zeta_inputs as zi
from oracle import cohomology

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "quintic_surfaces_r1.txt")


def test_surface_golden_shape_and_recipe():
    cases, cur = [], None
    for line in open(GOLDEN):
        if line.startswith("#") or ":" not in line:
            continue
        key, _, val = line.partition(":")
        if key.strip() == "case":
            cur = {"name": val.strip()}
            cases.append(cur)
        else:
            cur[key.strip()] = val.strip()
    assert [c["name"] for c in cases] == ["fermat", "quintic_surfaces_0"]
    want = {"fermat": zi.fermat(3, 5), "quintic_surfaces_0": zi.draw_instance("quintic_surfaces", 0,
                                                                               cohomology.is_smooth)[3]}
    for c in cases:
        assert c["n d p"] == "3 5 7" and int(c["q"]) == 7 ** 3
        assert [int(x) for x in c["coeffs"].split()] == list(want[c["name"]])
        Y = [int(x) for x in c["Y"].split()]
        assert len(Y) == 52 * 52 and all(0 <= y < 343 for y in Y) and any(Y)
