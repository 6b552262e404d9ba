"""Writes the stored expected values under tests/golden/ from the oracle alone.

Run from the repository root:  python tests/golden/make_golden.py
Each value is produced by oracle/ (which the point-count and closed-form
tests pin); nothing here touches the CUDA path.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import zeta_inputs as zi  # noqa: E402
from oracle import cohomology, zeta  # noqa: E402


def main():
    n, d, p, c, att = zi.draw_instance("quartic_curve_f11", 0, cohomology.is_smooth)
    res = zeta.compute_zeta(n, d, p, c)
    with open(os.path.join(HERE, "quartic_curve_f11.txt"), "w") as fh:
        fh.write("# dense plane quartic over F_11 (genus 3), seed 0; P(T) = det(1 - T F), Sec. 2.1\n")
        fh.write("# P(T) is also fixed by #X(F_11^r), r = 1..3 (tests/test_oracle_zeta.py)\n")
        fh.write("n d p: %d %d %d\n" % (n, d, p))
        fh.write("coeffs: %s\n" % " ".join(map(str, c)))
        fh.write("r_m N_m M: %s %s %d\n" % (" ".join("r%d=%d" % kv for kv in sorted(res.prec.r.items())),
                                          " ".join("N%d=%d" % kv for kv in sorted(res.prec.N.items())), res.prec.M))
        fh.write("P: %s\n" % " ".join(map(str, res.P)))


if __name__ == "__main__":
    main()
