"""GPU parity of the tensor-core path (exact limb-split modular GEMM steps, ZETA_PATH_GEMM).

The recurrence kernel is checked element by element against the oracle's Algorithm 2; whole
instances are checked against the oracle's columns Y and P(T), and against the CUDA-core path.
"""
import numpy as np
import pytest

import zeta_inputs as zi
from oracle import cohomology, pins, zeta as ozeta

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


def _instance(workload, i):
    n, d, p, c, _ = zi.draw_instance(workload, i, cohomology.is_smooth)
    return n, d, p, c


GEMM_CASES = [
    # (s, c, ks, moduli): the curve sizes (s = 28, 45), ragged s and c, one column, k = 0 and
    # k = 1, the largest s and c the path takes, moduli from 2^14 (3 digits) to 2^60 (8 digits)
    (28, 6, [5, 0, 1], [11 ** 8, 7 ** 16, 13 ** 15]),
    (45, 12, [9, 3, 40], [7 ** 16, 47 ** 10, 41 ** 11]),
    (45, 1, [1, 17], [47 ** 10, 3 ** 37]),
    (13, 3, [4, 2, 7, 1], [7 ** 5, 7 ** 20, 11 ** 17, 13 ** 16]),
    (64, 16, [6, 2], [(1 << 60) - 93, 2 ** 59 + 3]),
    (17, 9, [3, 5], [3 ** 37, 7 ** 5]),
    (33, 16, [12], [7 ** 4]),
]


def _problems(s, c, ks, qs, seed):
    count = len(ks)
    A = np.zeros((count, s, s), dtype=np.uint64)
    B = np.zeros((count, s, s), dtype=np.uint64)
    W = np.zeros((count, s, c), dtype=np.uint64)
    for t in range(count):
        A[t] = np.array(zi.random_residues(seed + t, s * s, qs[t]), dtype=np.uint64).reshape(s, s)
        B[t] = np.array(zi.random_residues(seed + 100 + t, s * s, qs[t]), dtype=np.uint64).reshape(s, s)
        W[t] = np.array(zi.random_residues(seed + 200 + t, s * c, qs[t]), dtype=np.uint64).reshape(s, c)
    return A, B, W


def _run(ctx, path, s, c, ks, qs, A, B, W):
    dev = lambda a: torch.from_numpy(a.view(np.int64).copy()).cuda()
    dA, dB, dW = dev(A), dev(B), dev(W)
    dk = torch.tensor(ks, dtype=torch.int32).cuda()
    dq = torch.tensor(np.array(qs, dtype=np.uint64).view(np.int64)).cuda()
    z.zeta_horner_device(ctx, path, len(ks), s, c, dk, dA, dB, dW, dq)
    torch.cuda.synchronize()
    return dW.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("s,c,ks,qs", GEMM_CASES)
def test_gemm_recurrence_matches_algorithm_2(ctx, s, c, ks, qs):
    A, B, W = _problems(s, c, ks, qs, 5000)
    out = _run(ctx, "gemm", s, c, ks, qs, A, B, W)
    for t in range(len(ks)):
        ref = ozeta.horner_python(A[t].astype(object), B[t].astype(object), W[t].astype(object), ks[t], qs[t])
        assert (out[t].astype(object) == ref).all(), (s, c, t)


def test_gemm_and_vector_recurrences_agree_on_many_problems(ctx):
    # 400 problems: more than one per SM, so blocks loop over problems and reuse their TMEM
    s, c = 45, 12
    primes = [7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47]
    qs = [p ** (12 + (t % 5)) for t, p in enumerate(primes * 34)][:400]
    qs = [q for q in qs if q < 1 << 60]
    ks = [1 + (t * 7) % 45 for t in range(len(qs))]
    A, B, W = _problems(s, c, ks, qs, 9000)
    g = _run(ctx, "gemm", s, c, ks, qs, A, B, W)
    v = _run(ctx, "vector", s, c, ks, qs, A, B, W)
    assert (g == v).all()
    ref = ozeta.horner_python(A[3].astype(object), B[3].astype(object), W[3].astype(object), ks[3], qs[3])
    assert (g[3].astype(object) == ref).all()


def test_gemm_path_rejects_sizes_it_does_not_take(ctx):
    dk = torch.zeros(1, dtype=torch.int32).cuda()
    buf = torch.zeros(1 << 16, dtype=torch.int64).cuda()
    dq = torch.tensor([7 ** 10], dtype=torch.int64).cuda()
    with pytest.raises(z.ZetaError):
        z.zeta_horner_device(ctx, "gemm", 1, 65, 4, dk, buf, buf, buf, dq)   # s > 64
    with pytest.raises(z.ZetaError):
        z.zeta_horner_device(ctx, "gemm", 1, 8, 17, dk, buf, buf, buf, dq)   # c > 16
    # a K3 surface (s = 220) is refused as a whole instance
    n, d, p, c = _instance("quartic_k3", 0)
    with pytest.raises(z.ZetaError):
        z.zeta_frobenius(ctx, (n, d, p, c), N=1, r=2, y_only=True, path="gemm")


def test_gemm_quartic_f11_matches_oracle(ctx):
    n, d, p, c = _instance("quartic_curve_f11", 0)
    ref = ozeta.compute_zeta(n, d, p, c)
    F, Y, st = z.zeta_frobenius(ctx, (n, d, p, c), path="gemm")
    assert (Y.astype(object) == ref.Y).all()
    assert (F.astype(object) == ref.F).all()
    P, _ = z.zeta_charpoly(ctx, (n, d, p, c), path="gemm")
    assert P == ref.P


@pytest.mark.parametrize("policy", ["p_chunk", "depth_first", "var_by_var"])
@pytest.mark.parametrize("i", [0, 11])
def test_gemm_quintic_columns_match_oracle(ctx, policy, i):
    n, d, p, c = _instance("quintic_curves", i)
    ref = ozeta.compute_zeta(n, d, p, c, policy="p_chunk")
    F, Y, _ = z.zeta_frobenius(ctx, (n, d, p, c), policy=policy, path="gemm")
    assert (Y.astype(object) == ref.Y).all()
    P, _ = z.zeta_charpoly(ctx, (n, d, p, c), policy=policy, path="gemm")
    assert P == ref.P


@pytest.mark.parametrize("n,d,p", [(2, 5, 11), (2, 4, 13), (2, 5, 41)])
def test_gemm_fermat_curves_closed_form(ctx, n, d, p):
    P, _ = z.zeta_charpoly(ctx, (n, d, p, zi.fermat(n, d)), path="gemm")
    assert P == pins.fermat_charpoly(n, d, p)


def test_gemm_batch_equals_vector_batch(ctx):
    # one persistent launch per path over 304 curves (two per SM), every prime of the workload
    specs = [_instance("quintic_curves", i) for i in range(304)]
    out_g, per_g, tot_g = z.zeta_batch(ctx, specs, policy="p_chunk", path="gemm")
    out_v, per_v, tot_v = z.zeta_batch(ctx, specs, policy="p_chunk", path="vector")
    assert all(x["status"] == 0 for x in per_g)
    assert out_g == out_v
    assert tot_g["column_steps"] == tot_v["column_steps"]
    for (n, d, p, c), P in zip(specs[:24], out_g[:24]):
        N1 = pins.count_points(n, d, p, c, 1)
        assert P[1] == pins.counts_to_charpoly_prefix(n, p, [N1])[1]
