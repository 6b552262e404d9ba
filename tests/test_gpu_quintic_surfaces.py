"""Quintic surfaces in P^3 (n = 3, d = 5: b = 52 basis columns, s = C(15, 3) = 455) at relative precision 1 on the
whole-GPU executor (the persistent executors carry at most 32 columns; the full precision, p^M = 7^49, needs
residues beyond 64 bits).  At r = 1 (M = 3) the library gives a_i mod p^(1 + H(i)), H the Hodge polygon (slope 0
four times, 1 on 44 columns, 2 four times): P(T) mod p, the unit-root part (and a_i mod p^min(1 + H(i), K), p^K the
largest power below 2^63).
 - The Fermat quintic surface: ordinary at 11 (p = 1 mod 5), where P(T) agrees with Weil's Gauss-sum formula
   modulo p^(1 + H(i)) in every coefficient and has four unit roots; no unit root at 7, 13 and 17, the primes at
   which the paper reports it supersingular.
 - Dense quintic surfaces over F_7 from the workload: P(T) mod p equals det(1 - T H) mod p for the Hasse-Witt
   matrix H (the oracle's closed form from the coefficients of f^(p-1)), with three policies.
"""
import pytest

import zeta_inputs as zi
from oracle import pins

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


def _accept(n, d, p, c):
    """Smooth (the full precision, p^M = 7^49, is refused: the query is made at relative precision 1)."""
    try:
        z.zeta_query((n, d, p, c), r=1)
        return True
    except z.ZetaError as e:
        if e.status == 2:
            return False
        raise


def test_fermat_quintic_surface_ordinary_at_11_supersingular_primes_have_no_unit_root(ctx):
    from paper_2602_24155_gb300.newton import hodge_polygon, unit_roots_mod_p
    n, d = 3, 5
    specs = [(n, d, p, zi.fermat(n, d)) for p in (7, 11, 13, 17)]
    P, per, tot = z.zeta_batch(ctx, specs, policy="p_chunk", r=1)
    assert [st["status"] for st in per] == [0] * 4
    assert all(st["b"] == 52 and st["s"] == 455 for st in per)
    exact = pins.fermat_charpoly(n, d, 11, dps=200)
    H = hodge_polygon(n, d)
    K = max(k for k in range(64) if 11 ** k < 2 ** 63)   # the finish works mod the largest power below 2^63
    for i in range(1, 27):
        assert (P[1][i] - exact[i]) % 11 ** min(1 + H[i], K) == 0, i
    assert [unit_roots_mod_p(Pi, p) for Pi, p in zip(P, (7, 11, 13, 17))] == [0, 4, 0, 0]
    print("Fermat quintic surface at 7, 11, 13, 17, r = 1: %d steps, %.0f ms of kernels in %d launches"
          % (tot["steps"], tot["ms_kernel"], tot["kernel_launches"]))


def test_dense_quintic_surfaces_equal_hasse_witt(ctx):
    specs = [zi.draw_instance("quintic_surfaces", i, _accept)[:4] for i in range(6)]
    out = {}
    for policy in ("p_chunk", "cover", "depth_first"):
        P, per, tot = z.zeta_batch(ctx, specs, policy=policy, r=1)
        assert [st["status"] for st in per] == [0] * len(specs)
        out[policy] = [[a % 7 for a in Pi] for Pi in P]
        print("6 dense quintic surfaces over F_7, r = 1, %s: %d column steps, %.0f ms of kernels"
              % (policy, tot["column_steps"], tot["ms_kernel"]))
    for i, (n, d, p, c) in enumerate(specs):
        hw = pins.hasse_witt_charpoly_mod_p(n, d, p, c)
        want = [(hw[t] if t < len(hw) else 0) % p for t in range(53)]
        for policy in out:
            assert out[policy][i] == want, (i, policy)


def _surface_golden():
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "quintic_surfaces_r1.txt")
    cases, cur = [], None
    for line in open(path):
        if line.startswith("#") or ":" not in line:
            continue
        key, _, val = line.partition(":")
        key, val = key.strip(), val.strip()
        if key == "case":
            cur = {"name": val}
            cases.append(cur)
        else:
            cur[key] = val
    return cases


def test_quintic_surface_Y_equals_the_oracle(ctx):
    """The unnormalised Frobenius columns Y (52 x 52 mod 7^3) of the Fermat quintic surface and a dense one over F_7
    at relative precision 1, through the single-instance call on the whole-GPU executor, equal the oracle's
    (tests/golden/quintic_surfaces_r1.txt, written by make_golden.py surface from the oracle alone), for two
    policies (Y depends on neither the policy nor S)."""
    import numpy as np
    for case in _surface_golden():
        n, d, p = map(int, case["n d p"].split())
        c = [int(x) for x in case["coeffs"].split()]
        want = np.array([int(x) for x in case["Y"].split()], dtype=object).reshape(52, 52)
        for policy in ("p_chunk", "cover"):
            F, Y, st = z.zeta_frobenius(ctx, (n, d, p, c), r=1, y_only=True, policy=policy)
            assert st["b"] == 52 and st["s"] == 455
            assert (Y.astype(object) == want).all(), (case["name"], policy)
