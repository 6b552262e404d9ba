"""A dense cubic fourfold over F_7 (s = 3003, b = 22, S = {5}) at relative precision 1 on the whole-GPU executor.

The full P(T) needs residues mod 7^25 (beyond 64-bit words) and is out of the oracle's reach at s = 3003; at
relative precision 1 (M = 9) the library determines a_i mod p^(1 + H(i)), H the Hodge polygon (0, 1, 3, 5, ...),
which is what the Newton height needs (a cubic fourfold's primitive H^4 has a K3 surface's Hodge shape raised by
one: its first slope is 2 - 1/h).  The pins come from point counts (tests/golden/cubic_fourfold_f7.txt, written
by make_golden.py fourfold from the oracle's point counting): #X(F_7) and #X(F_49) fix tr F and tr F^2, hence a_1
and a_2 exactly (Newton's identities); the GPU's a_1 must agree mod 7^2 and a_2 mod 7^4.
"""
import os

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
z = pytest.importorskip("paper_2602_24155_gb300")

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


def test_dense_cubic_fourfold_f7_against_point_counts():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2602_24155_gb300.newton import fourfold_height
    n, d, p, c, (N1, N2) = _golden()
    ctx = z.zeta_create(0, torch.cuda.current_stream().cuda_stream)
    try:
        P, per, tot = z.zeta_batch(ctx, [(n, d, p, c)], policy="p_chunk", r=1)
    finally:
        z.zeta_destroy(ctx)
    st = per[0]
    print("dense cubic fourfold over F_7, r = 1: %d chunks, %d steps, %d column steps; setup %.0f ms, kernels %.0f ms "
          "in %d launches; height %s" % (tot["chunks"], tot["steps"], tot["column_steps"], tot["ms_host_setup"],
                                         tot["ms_kernel"], tot["kernel_launches"], fourfold_height(P[0], p)))
    assert st["status"] == 0 and st["s"] == 3003 and st["b"] == 22 and st["M"] == 9
    s1 = N1 - sum(p ** i for i in range(n))            # tr F on primitive H^4
    s2 = N2 - sum(p ** (2 * i) for i in range(n))      # tr F^2
    a1, a2 = -s1, (s1 * s1 - s2) // 2
    assert (s1 * s1 - s2) % 2 == 0
    assert (P[0][1] - a1) % p ** 2 == 0
    assert (P[0][2] - a2) % p ** 4 == 0
