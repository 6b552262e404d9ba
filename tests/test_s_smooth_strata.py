"""The library's S-smoothness test (coordinate strata: a square system of restricted partial derivatives per
stratum, each decided by Macaulay's criterion) against the oracle's (the map of J_S onto Homog_kappa,
Definition 3.1 read through Macaulay).  Both decide whether the J_S generators have a common zero; they must agree
on every instance, smooth or not, for one- and two-element S."""
import pytest

import zeta_inputs as zi
from oracle import cohomology

z = pytest.importorskip("paper_2602_24155_gb300")


def _lib_status(spec, S):
    try:
        z.zeta_query(spec, S=S)
        return 0
    except z.ZetaError as e:
        return e.status


@pytest.mark.parametrize("n,d,p,S,count", [(2, 3, 7, (2,), 60), (3, 3, 7, (3,), 60), (3, 3, 11, (0,), 30),
                                           (3, 3, 13, (1, 3), 30)])
def test_strata_agree_with_the_oracle(n, d, p, S, count):
    kinds = set()
    for i in range(count):
        c = zi.dense_candidate(n, d, p, 77, i, 0)
        smooth = cohomology.is_smooth(n, d, p, c)
        want = 0 if smooth and cohomology.is_S_smooth(n, d, p, c, S) else 2
        assert _lib_status((n, d, p, c), list(S)) == want, (n, d, p, S, i)
        kinds.add((smooth, want))
    assert (True, 0) in kinds and (True, 2) in kinds   # both verdicts occur among smooth instances
