"""Writes the stored expected values under tests/golden/ from the oracle alone.

Run from the repository root:  python tests/golden/make_golden.py [k3 | threefold | fourfold | surface]
Each value is produced by oracle/ (which the point-count and closed-form
tests pin); nothing here touches the CUDA path.  `k3` writes the
full-precision P(T) of three quartic K3 surfaces (tens of minutes of CPU per
surface, one process each).  `threefold` writes P(T) of the dense cubic
threefold over F_11 drawn with seed 11 (S = {4}) at series order N = 6, the
least N whose columns reach the relative precision r = (5, 6) (about half an
hour of CPU).  `fourfold` writes #X(F_7) and #X(F_49) of a dense cubic
fourfold (point counts, about ten minutes of CPU): its P(T) is beyond the
oracle's reach (s = 3003), the counts fix a_1 and a_2.  `surface` writes the
unnormalised Frobenius columns Y of quintic surfaces at relative precision 1
(b = 52, Y mod 7^3; about a minute of CPU each).
"""
import multiprocessing as mp
import os
import sys
import time

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


# quartic K3 workload members with their character: sparse over F_7, dense over F_13, dense over F_7
K3_GOLDEN = [9, 2, 0]


def _k3_one(i):
    n, d, p, c, att = zi.draw_instance("quartic_k3", i, cohomology.is_smooth)
    t = time.time()
    res = zeta.compute_zeta(n, d, p, c, policy="p_chunk")
    return i, n, d, p, c, res.prec, [int(x) for x in res.P], time.time() - t


def k3_main():
    with mp.get_context("spawn").Pool(len(K3_GOLDEN)) as pool:
        rows = pool.map(_k3_one, K3_GOLDEN)
    with open(os.path.join(HERE, "quartic_k3_full.txt"), "w") as fh:
        fh.write("# quartic K3 surfaces of the quartic_k3 workload (seed 2) at the full precision of the oracle's\n")
        fh.write("# rules (r_m, N_m, M); P(T) = det(1 - T F) of degree 21, Sec. 2.1; written by make_golden.py k3\n")
        for i, n, d, p, c, prec, P, secs in rows:
            fh.write("instance: %d\n" % i)
            fh.write("n d p: %d %d %d\n" % (n, d, p))
            fh.write("coeffs: %s\n" % " ".join(map(str, c)))
            fh.write("r_m N_m M: %s %s %d\n" % (" ".join("r%d=%d" % kv for kv in sorted(prec.r.items())),
                                              " ".join("N%d=%d" % kv for kv in sorted(prec.N.items())), prec.M))
            fh.write("oracle seconds: %.0f\n" % secs)
            fh.write("P: %s\n" % " ".join(map(str, P)))


def threefold_main():
    n, d, p = 4, 3, 11
    att = 0
    while True:
        c = zi.dense_candidate(n, d, p, 11, 0, att)
        att += 1
        if cohomology.is_smooth(n, d, p, c) and cohomology.is_S_smooth(n, d, p, c, (4,)):
            break
    t = time.time()
    res = zeta.compute_zeta(n, d, p, c, policy="p_chunk", S=(4,), N=6)
    with open(os.path.join(HERE, "cubic_threefold_f11.txt"), "w") as fh:
        fh.write("# dense cubic threefold over F_11 (zeta_inputs.dense_candidate seed 11, instance 0, first smooth and\n")
        fh.write("# {4}-smooth attempt), reduction with S = {4}; P(T) = det(1 - T F) of degree 10, Sec. 2.1\n")
        fh.write("# series order N = 6 (mod 11^11): the columns reach r = (5, 6); N = 5 lifts to the same P(T)\n")
        fh.write("n d p: %d %d %d\n" % (n, d, p))
        fh.write("coeffs: %s\n" % " ".join(map(str, c)))
        fh.write("M: %d\n" % res.prec.M)
        fh.write("oracle seconds: %.0f\n" % (time.time() - t))
        fh.write("P: %s\n" % " ".join(map(str, res.P)))


# dense_candidate(5, 3, 7, seed 5, instance i, attempt 0) for i = 0, 1, ...: about one draw in sixty is
# {5}-smooth over F_7 (a common zero of the J_S generators may sit on any of 32 coordinate strata); instance 76 is
# the first
FOURFOLD_INSTANCE = 76


def fourfold_main():
    from oracle import pins
    n, d, p = 5, 3, 7
    c = zi.dense_candidate(n, d, p, 5, FOURFOLD_INSTANCE, 0)
    assert cohomology.is_smooth(n, d, p, c)
    t = time.time()
    counts = [pins.count_points(n, d, p, c, r) for r in (1, 2)]
    with open(os.path.join(HERE, "cubic_fourfold_f7.txt"), "w") as fh:
        fh.write("# dense cubic fourfold over F_7 (zeta_inputs.dense_candidate seed 5, instance %d, attempt 0),\n"
                 % FOURFOLD_INSTANCE)
        fh.write("# smooth and {5}-smooth; #X(F_7^r) for r = 1, 2 by evaluating f on every point of P^5\n")
        fh.write("n d p: %d %d %d\n" % (n, d, p))
        fh.write("coeffs: %s\n" % " ".join(map(str, c)))
        fh.write("oracle seconds: %.0f\n" % (time.time() - t))
        fh.write("counts: %s\n" % " ".join(map(str, counts)))


def surface_main():
    """Y (52 x 52, mod q = p^M, unnormalised) of quintic surfaces at relative precision r = 1: the Fermat quintic
    surface over F_7 and the first dense surface of the quintic_surfaces workload."""
    n, d, p = 3, 5, 7
    cases = [("fermat", zi.fermat(n, d)),
             ("quintic_surfaces_0", zi.draw_instance("quintic_surfaces", 0, cohomology.is_smooth)[3])]
    with open(os.path.join(HERE, "quintic_surfaces_r1.txt"), "w") as fh:
        fh.write("# quintic surfaces over F_7 at relative precision r = 1: Y = unnormalised Frobenius columns\n")
        fh.write("# (b x b, row-major, mod q), the same for every policy and every S\n")
        for name, c in cases:
            t = time.time()
            res = zeta.compute_zeta(n, d, p, c, r=1, normalise=False, want_P=False)
            fh.write("case: %s\n" % name)
            fh.write("n d p: %d %d %d\n" % (n, d, p))
            fh.write("coeffs: %s\n" % " ".join(map(str, c)))
            fh.write("q: %d\n" % res.prec.q)
            fh.write("oracle seconds: %.0f\n" % (time.time() - t))
            fh.write("Y: %s\n" % " ".join(str(int(v)) for v in res.Y.reshape(-1)))


if __name__ == "__main__":
    if len(sys.argv) > 1 and sys.argv[1] == "k3":
        k3_main()
    elif len(sys.argv) > 1 and sys.argv[1] == "threefold":
        threefold_main()
    elif len(sys.argv) > 1 and sys.argv[1] == "fourfold":
        fourfold_main()
    elif len(sys.argv) > 1 and sys.argv[1] == "surface":
        surface_main()
    else:
        main()
