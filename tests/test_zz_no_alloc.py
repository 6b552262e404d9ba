"""The allocation-free entry point (zeta_horner_static) against zeta_horner_device and Algorithm 2.

zeta_horner_static serves callers that may not allocate device memory (a
framework's memory pool or budget, plugins that must not call cudaMalloc
after start-up): its matrix scratch is a 16 MiB array compiled into the
library.  These checks compare it with the context-based entry point on the
same inputs, bit for bit, on two calls in a row (the second call reuses the
array the first one left behind), check one case directly against the
oracle's Algorithm 2, check that a bad modulus is reported without touching
that problem's W while the others are computed, and check that oversize
problems are refused before anything runs.  This file is collected last on
purpose.
"""
import numpy as np
import pytest

import zeta_inputs as zi
from oracle.zeta import horner_python

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
z = pytest.importorskip("paper_2602_24155_gb300")


def _problems(seed, count, s, c, ks, qs):
    A = np.zeros((count, s, s), dtype=np.uint64)
    B = np.zeros((count, s, s), dtype=np.uint64)
    W = np.zeros((count, s, c), dtype=np.uint64)
    for t in range(count):
        A[t] = np.array(zi.random_residues(seed + 10 * t, s * s, qs[t]), dtype=np.uint64).reshape(s, s)
        B[t] = np.array(zi.random_residues(seed + 10 * t + 1, s * s, qs[t]), dtype=np.uint64).reshape(s, s)
        W[t] = np.array(zi.random_residues(seed + 10 * t + 2, s * c, qs[t]), dtype=np.uint64).reshape(s, c)
    dev = lambda a: torch.from_numpy(a.view(np.int64)).cuda()
    k = torch.tensor(ks, dtype=torch.int32).cuda()
    q = torch.tensor(np.array(qs, dtype=np.uint64).view(np.int64)).cuda()
    return dev(A), dev(B), dev(W), k, q


def test_static_entry_matches_the_context_entry_twice():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    stream = torch.cuda.current_stream()
    ctx = z.zeta_create(0, stream.cuda_stream)
    try:
        cases = [
            # (seed, s, c, ks, qs): K3-sized matrices, then quintic-curve-sized ones
            (11, 220, 21, [3, 0, 5], [7 ** 20, 11 ** 16, 13 ** 14]),
            (29, 45, 12, [9, 1, 4, 7, 2, 6, 3, 8], [7 ** 15, 47 ** 9, 41 ** 11, 13 ** 11, 3 ** 30, 7 ** 16, 11 ** 13, 2 ** 59 + 1]),
        ]
        for seed, s, c, ks, qs in cases:
            A, B, W, k, q = _problems(seed, len(ks), s, c, ks, qs)
            W_ref = W.clone()
            z.zeta_horner_device(ctx, "vector", len(ks), s, c, k, A, B, W_ref, q)
            z.zeta_horner_static(stream.cuda_stream, len(ks), s, c, k, A, B, W, q)
            torch.cuda.synchronize()
            assert torch.equal(W, W_ref), (s, c)
    finally:
        z.zeta_destroy(ctx)


def test_static_entry_refuses_oversize_problems():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    buf = torch.zeros(16, dtype=torch.int64).cuda()
    k = torch.zeros(1, dtype=torch.int32).cuda()
    with pytest.raises(z.ZetaError) as e:
        z.zeta_horner_static(None, 1, 600, 4, k, buf, buf, buf, buf)    # s > 512
    assert e.value.status == 1
    with pytest.raises(z.ZetaError) as e:
        z.zeta_horner_static(None, 1, 8, 40, k, buf, buf, buf, buf)     # c > 32
    assert e.value.status == 1


def test_static_entry_matches_algorithm_2_of_the_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    stream = torch.cuda.current_stream()
    s, c, ks, qs = 28, 6, [4, 7], [11 ** 7, 41 ** 11]
    A, B, W, k, q = _problems(5, len(ks), s, c, ks, qs)
    A_h, B_h, W_h = (x.cpu().numpy().view(np.uint64) for x in (A, B, W))
    z.zeta_horner_static(stream.cuda_stream, len(ks), s, c, k, A, B, W, q)
    torch.cuda.synchronize()
    out = W.cpu().numpy().view(np.uint64)
    for t in range(len(ks)):
        obj = lambda a: np.array([[int(x) for x in row] for row in a], dtype=object)
        ref = horner_python(obj(A_h[t]), obj(B_h[t]), obj(W_h[t]), ks[t], qs[t])
        assert [[int(x) for x in row] for row in out[t]] == [[int(x) for x in row] for row in ref], t


def test_static_entry_reports_a_bad_modulus_and_computes_the_rest():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    stream = torch.cuda.current_stream()
    ctx = z.zeta_create(0, stream.cuda_stream)
    try:
        s, c, ks = 45, 8, [3, 5, 2]
        qs = [13 ** 11, 7 ** 15, 11 ** 13]
        A, B, W, k, q = _problems(41, len(ks), s, c, ks, qs)
        W_ref = W.clone()
        z.zeta_horner_device(ctx, "vector", len(ks), s, c, k, A, B, W_ref, q)
        W_before = W.clone()
        q_bad = q.clone()
        q_bad[1] = 2 * 7 ** 15              # even modulus for problem 1 only
        with pytest.raises(z.ZetaError) as e:
            z.zeta_horner_static(stream.cuda_stream, len(ks), s, c, k, A, B, W, q_bad)
        assert e.value.status == 1
        torch.cuda.synchronize()
        assert torch.equal(W[1], W_before[1])       # the refused problem is untouched
        assert torch.equal(W[0], W_ref[0]) and torch.equal(W[2], W_ref[2])
        W2 = W_before.clone()
        z.zeta_horner_static(stream.cuda_stream, len(ks), s, c, k, A, B, W2, q)   # status cleared: ZETA_OK
        torch.cuda.synchronize()
        assert torch.equal(W2, W_ref)
    finally:
        z.zeta_destroy(ctx)
