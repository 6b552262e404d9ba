"""The stored point counts of the dense cubic fourfold over F_7 (tests/golden/cubic_fourfold_f7.txt).

They pin the GPU's a_1 and a_2 (tests/test_gpu_fourfold.py).  Checked here on the CPU: the coefficients are the
stated draw and define a smooth fourfold, #X(F_7) recounts to the stored value, and both traces of Frobenius on the
22-dimensional primitive H^4 obey the Weil bound |tr F^r| <= 22 p^(2r).
"""
import os

import zeta_inputs as zi
from oracle import cohomology, pins

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cubic_fourfold_f7.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or ":" not in line:
            continue
        key, _, val = line.partition(":")
        out[key.strip()] = val.strip()
    n, d, p = map(int, out["n d p"].split())
    return n, d, p, [int(x) for x in out["coeffs"].split()], [int(x) for x in out["counts"].split()]


def test_fourfold_golden_counts():
    n, d, p, c, counts = _golden()
    assert (n, d, p) == (5, 3, 7)
    assert c == zi.dense_candidate(5, 3, 7, 5, 76, 0)
    assert cohomology.is_smooth(n, d, p, c)
    assert pins.count_points(n, d, p, c, 1) == counts[0]
    for r, N in enumerate(counts, start=1):
        tr = N - sum(p ** (r * i) for i in range(n))
        assert abs(tr) <= 22 * p ** (2 * r)
