"""GPU parity: the CUDA path through the C ABI against the oracle (bit-exact)."""
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


HORNER_CASES = [
    # (s, c, ks, moduli): ragged s (not a multiple of 4), one column, k = 0 and k = 1
    (28, 6, [5, 0, 1], [11 ** 8, 7 ** 16, 13 ** 15]),
    (45, 12, [9, 3], [7 ** 16, 47 ** 10]),
    (45, 1, [1, 17], [47 ** 10, 3 ** 37]),
    (13, 3, [4, 2, 7, 1], [7 ** 5, 7 ** 20, 11 ** 17, 13 ** 16]),
    (220, 21, [3], [7 ** 20]),
    (67, 7, [4, 6], [13 ** 15, 2 ** 59 + 3]),
]


@pytest.mark.parametrize("s,c,ks,qs", HORNER_CASES)
def test_horner_kernel_matches_algorithm_2(ctx, s, c, ks, qs):
    count = len(ks)
    A = np.zeros((count, s, s), dtype=np.uint64)
    B = np.zeros((count, s, s), dtype=np.uint64)
    W = np.zeros((count, s, c), dtype=np.uint64)
    for t in range(count):
        A[t] = np.array(zi.random_residues(1000 + t, s * s, qs[t]), dtype=np.uint64).reshape(s, s)
        B[t] = np.array(zi.random_residues(2000 + t, s * s, qs[t]), dtype=np.uint64).reshape(s, s)
        W[t] = np.array(zi.random_residues(3000 + t, s * c, qs[t]), dtype=np.uint64).reshape(s, c)
    dev = lambda a: torch.from_numpy(a.view(np.int64)).cuda()
    dA, dB, dW = dev(A), dev(B), dev(W)
    dk = torch.tensor(ks, dtype=torch.int32).cuda()
    dq = torch.tensor(np.array(qs, dtype=np.uint64).view(np.int64)).cuda()
    z.zeta_horner_device(ctx, "vector", count, s, c, dk, dA, dB, dW, dq)
    torch.cuda.synchronize()
    out = dW.cpu().numpy().view(np.uint64)
    for t in range(count):
        ref = ozeta.horner_python(A[t].astype(object), B[t].astype(object), W[t].astype(object), ks[t], qs[t])
        assert (out[t].astype(object) == ref).all(), (s, c, t)


def test_horner_kernel_rejects_bad_sizes(ctx):
    dk = torch.zeros(1, dtype=torch.int32).cuda()
    buf = torch.zeros(1024 * 1024, dtype=torch.int64).cuda()
    dq = torch.tensor([7 ** 10], dtype=torch.int64).cuda()
    with pytest.raises(z.ZetaError):
        z.zeta_horner_device(ctx, "vector", 1, 600, 4, dk, buf, buf, buf, dq)   # s > 512
    with pytest.raises(z.ZetaError):
        z.zeta_horner_device(ctx, "vector", 1, 8, 40, dk, buf, buf, buf, dq)    # c > 32
    dq2 = torch.tensor([1 << 40], dtype=torch.int64).cuda()                      # even modulus
    with pytest.raises(z.ZetaError):
        z.zeta_horner_device(ctx, "vector", 1, 8, 4, dk, buf, buf, buf, dq2)


@pytest.fixture(scope="module")
def quartic_ref():
    n, d, p, c = _instance("quartic_curve_f11", 0)
    return (n, d, p, c), ozeta.compute_zeta(n, d, p, c)


def test_quartic_f11_frobenius_and_charpoly(ctx, quartic_ref):
    spec, ref = quartic_ref
    F, Y, st = z.zeta_frobenius(ctx, spec)
    assert (Y.astype(object) == ref.Y).all()
    assert (F.astype(object) == ref.F).all()
    P, st = z.zeta_charpoly(ctx, spec)
    assert P == ref.P
    assert st["b"] == 6 and st["M"] == ref.prec.M and st["r"] == max(ref.prec.r.values())


@pytest.mark.parametrize("i", [0, 1, 2])
def test_quintic_curves_match_oracle(ctx, i):
    n, d, p, c = _instance("quintic_curves", i)
    ref = ozeta.compute_zeta(n, d, p, c)
    F, Y, _ = z.zeta_frobenius(ctx, (n, d, p, c))
    assert (Y.astype(object) == ref.Y).all()
    P, _ = z.zeta_charpoly(ctx, (n, d, p, c))
    assert P == ref.P


@pytest.mark.parametrize("policy", ["p_chunk", "var_by_var", "depth_first"])
@pytest.mark.parametrize("which", [("quartic_curve_f11", 0), ("quintic_curves", 0), ("quintic_curves", 11)])
def test_policies_reach_the_same_columns(ctx, policy, which):
    # Y depends only on the basis, N_m and M: every policy must reproduce the oracle's
    n, d, p, c = _instance(*which)
    ref = ozeta.compute_zeta(n, d, p, c, policy="p_chunk" if which[1] == 11 else "depth_first")
    F, Y, st = z.zeta_frobenius(ctx, (n, d, p, c), policy=policy)
    assert (Y.astype(object) == ref.Y).all()
    P, _ = z.zeta_charpoly(ctx, (n, d, p, c), policy=policy)
    assert P == ref.P
    if policy == "p_chunk":
        assert st["column_steps"] == ref.log.column_steps if which[1] == 11 else True


@pytest.mark.parametrize("n,d,p", [(2, 5, 11), (2, 4, 13), (2, 5, 31)])
def test_fermat_curves_closed_form_on_gpu(ctx, n, d, p):
    P, _ = z.zeta_charpoly(ctx, (n, d, p, zi.fermat(n, d)))
    assert P == pins.fermat_charpoly(n, d, p)


@pytest.mark.parametrize("N", [1, {1: 2, 2: 1, 3: 1}])
def test_k3_truncated_unnormalised_columns(ctx, N):
    # quartic K3 surface (s = 220, b = 21) at a truncated series order: Y only
    n, d, p, c = _instance("quartic_k3", 0)
    ref = ozeta.compute_zeta(n, d, p, c, N=N, r=2, normalise=False)
    F, Y, st = z.zeta_frobenius(ctx, (n, d, p, c), N=N, r=2, y_only=True)
    assert st["s"] == 220 and st["b"] == 21
    assert (Y.astype(object) == ref.Y).all()


def test_batch_matches_single_calls_and_phases(ctx, quartic_ref):
    specs = [quartic_ref[0], _instance("quintic_curves", 1), (2, 5, 11, zi.fermat(2, 5)), _instance("quintic_curves", 0)]
    singles = [z.zeta_charpoly(ctx, s)[0] for s in specs]
    out, per, total = z.zeta_batch(ctx, specs)
    assert out == singles
    assert all(x["status"] == 0 for x in per)
    assert total["column_steps"] > 0
    plan = z.zeta_batch_prepare(ctx, specs)
    plan.run()
    plan.run()
    out2, _, _ = plan.finish()
    plan.release()
    assert out2 == singles


def test_batch_reports_bad_instances(ctx):
    bad = [1 if m in [(4, 0, 0), (0, 4, 0)] else 0 for m in
           __import__("oracle.algebra", fromlist=["monomials"]).monomials(3, 4)]
    specs = [(2, 4, 7, bad), (2, 4, 13, zi.fermat(2, 4))]
    out, per, _ = z.zeta_batch(ctx, specs)
    assert out[0] is None and per[0]["status"] == 2
    assert out[1] == pins.fermat_charpoly(2, 4, 13)


def test_full_quintic_workload_sampled_parity(ctx):
    """The bench's workload (4096 plane quintics over 12 primes) in its launch configuration:
    every P(T) checked against a point count over F_p and Weil's bound; a sample against the oracle."""
    count = zi.WORKLOADS["quintic_curves"]["count"]
    specs = [_instance("quintic_curves", i) for i in range(count)]
    out, per, total = z.zeta_batch(ctx, specs, policy="p_chunk")
    assert all(P is not None for P in out)
    for (n, d, p, c), P in zip(specs, out):
        assert P[0] == 1 and len(P) == 13
        N1 = pins.count_points(n, d, p, c, 1)
        assert P[1] == pins.counts_to_charpoly_prefix(n, p, [N1])[1]
        alphas = np.roots(np.array(P, dtype=float))   # roots of sum a_i T^{b-i}: the alpha_j
        assert np.allclose(np.abs(alphas), np.sqrt(p), rtol=1e-6)
    for i in (0, 1, 2, 1000):
        n, d, p, c = specs[i]
        if p > 13:
            continue
        ref = ozeta.compute_zeta(n, d, p, c)
        assert out[i] == ref.P


def test_mixed_degrees_in_one_launch(ctx):
    # plane quartics (s = 28, b = 6) and quintics (s = 45, b = 12) over several primes in one persistent launch
    specs = [_instance("quartic_curve_f11", i) for i in range(6)] + [_instance("quintic_curves", i) for i in range(26)]
    out, per, total = z.zeta_batch(ctx, specs, policy="p_chunk")
    assert total["kernel_launches"] == 1
    for i in (0, 5, 6, 31):
        assert out[i] == z.zeta_charpoly(ctx, specs[i], policy="p_chunk")[0]
    assert out[0] == ozeta.compute_zeta(*specs[0]).P
    assert all(x["status"] == 0 for x in per)


@pytest.mark.parametrize("which", [("quartic_curve_f11", 0), ("quintic_curves", 0), ("quintic_curves", 11)])
def test_cover_policy_matches_oracle(ctx, which):
    n, d, p, c = _instance(*which)
    ref = ozeta.compute_zeta(n, d, p, c, policy="p_chunk")
    F, Y, st = z.zeta_frobenius(ctx, (n, d, p, c), policy="cover")
    assert (Y.astype(object) == ref.Y).all()
    assert z.zeta_charpoly(ctx, (n, d, p, c), policy="cover")[0] == ref.P


def test_cover_batch_equals_p_chunk_batch(ctx):
    specs = [_instance("quintic_curves", i) for i in range(304)]
    out_c, per_c, tot_c = z.zeta_batch(ctx, specs, policy="cover")
    out_p, per_p, tot_p = z.zeta_batch(ctx, specs, policy="p_chunk")
    assert out_c == out_p
    assert tot_c["column_steps"] < 0.85 * tot_p["column_steps"]
