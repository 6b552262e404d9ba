"""Learned direction policy: the network's gradients and scores against a float64 oracle, the training
data generated by rollouts of the game, the gain of the trained network over the method without it (the
cover game with Algorithm 3), and the learned policy's P(T) against the oracle."""
import numpy as np
import pytest

import zeta_inputs as zi
from oracle import cohomology, mlp as omlp, zeta as ozeta

z = pytest.importorskip("paper_2602_24155_gb300")


def _instance(workload, i):
    n, d, p, c, _ = zi.draw_instance(workload, i, cohomology.is_smooth)
    return n, d, p, c


def test_oracle_network_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    H = 8
    P = omlp.F * H + H + H * H + H + H + 1
    params = rng.normal(0, 0.5, P)
    X = rng.normal(0, 1, (11, omlp.F))
    go = np.array([0, 3, 7, 11])
    lab = np.array([1, 0, 3])
    loss, grad = omlp.loss_and_grad(params, H, X, go, lab)
    eps = 1e-6
    for k in rng.choice(P, 25, replace=False):
        e = np.zeros(P)
        e[k] = eps
        num = (omlp.loss_and_grad(params + e, H, X, go, lab)[0] - omlp.loss_and_grad(params - e, H, X, go, lab)[0]) / (2 * eps)
        assert abs(num - grad[k]) < 1e-6 * max(1.0, abs(num))


def test_dataset_is_generated_by_the_game():
    spec = _instance("quintic_curves", 0)
    X, go, lab, cost = z.zeta_policy_dataset(spec)
    assert X.shape[1] == z.POLICY_FEATURES and len(go) == len(lab) + 1
    assert 0 < len(lab) <= 128                                        # a sample of the decisions
    for g in range(len(lab)):
        a, b = go[g], go[g + 1]
        assert b - a >= 2
        assert X[a, 14] == 1.0 and (X[a + 1:b, 14] == 0.0).all()   # row 0 is Algorithm 3's choice
        assert cost[a + lab[g]] == 0 and (cost[a:b] >= 0).all()       # the label is the cheapest rollout
        assert lab[g] == 0 or cost[a] > 0                             # ties go to Algorithm 3
        assert ((X[a:b, 16] == 1.0) == (X[a:b, 15] > 0)).all()        # merge indicator agrees with the count
    # the two-call protocol returns the same data as a fresh call
    X2, go2, lab2, cost2 = z.zeta_policy_dataset(spec)
    assert (X2 == X).all() and (lab2 == lab).all() and (cost2 == cost).all()


def test_host_scores_match_the_oracle_network():
    # the forward pass the scheduler runs (host) against the float64 oracle
    rng = np.random.default_rng(3)
    for H in (4, 8, 64):
        w = z.zeta_mlp_init(H, 11)
        X = rng.normal(0, 1, (300, z.POLICY_FEATURES)).astype(np.float32)
        s = z.zeta_mlp_forward_host(H, w, X)
        ref = omlp.forward(w.astype(np.float64), H, X.astype(np.float64))[0]
        assert np.allclose(s, ref, rtol=1e-4, atol=1e-5)


def test_learned_policy_without_weights_plays_p_chunk():
    spec = _instance("quintic_curves", 3)
    a = z.zeta_plan(spec, policy="p_chunk")["game"]
    b = z.zeta_plan(spec, policy="learned")["game"]
    assert a == b


@pytest.mark.gpu
def test_gpu_network_gradient_matches_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    ctx = z.zeta_create(0)
    try:
        spec = _instance("quintic_curves", 1)
        X, go, lab, _ = z.zeta_policy_dataset(spec)
        ng = min(100, len(lab))
        X, go, lab = X[:go[ng]], go[:ng + 1], lab[:ng]
        for H in (16, 64, 128):
            w = z.zeta_mlp_init(H, 7)
            g, loss = z.zeta_mlp_grad(ctx, H, w, X, go, lab)
            ref_loss, ref_g = omlp.loss_and_grad(w.astype(np.float64), H, X.astype(np.float64), go, lab)
            assert abs(loss - ref_loss) < 1e-4 * max(1, abs(ref_loss))
            assert np.allclose(g, ref_g, rtol=1e-3, atol=1e-5)
            s = z.zeta_mlp_forward(ctx, H, w, X)
            assert np.allclose(s, omlp.forward(w, H, X)[0], rtol=1e-4, atol=1e-5)
    finally:
        z.zeta_destroy(ctx)


def _game_cost(g):
    # the cost the rollouts minimise: column steps plus 10 per chunk (zeta_policy_dataset)
    return g["column_steps"] + 10 * g["chunks"]


@pytest.mark.gpu
def test_trained_policy_gains_over_the_method_without_it():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2602_24155_gb300.policy_train import train_policy
    ctx = z.zeta_create(0)
    try:
        train = [_instance("quintic_curves", i) for i in range(12, 12 + 48)]
        held = [_instance("quintic_curves", i) for i in range(12)]
        w, loss, nd = train_policy(ctx, train, hidden=8, epochs=30)
        assert nd > 1000
        # the method without the network: the same cover levels with Algorithm 3's directions
        cover = sum(_game_cost(z.zeta_plan(s, policy="cover")["game"]) for s in held)
        learned = sum(_game_cost(z.zeta_plan(s, policy="learned", weights=w, hidden=8)["game"]) for s in held)
        pchunk = sum(_game_cost(z.zeta_plan(s, policy="p_chunk")["game"]) for s in held)
        print("game cost over 12 held-out quintic curves: p-chunk %d, cover %d, learned %d (network gain %.2f%%)"
              % (pchunk, cover, learned, 100.0 * (1 - learned / cover)))
        assert learned < cover, (learned, cover)
        for s in held[:3]:
            P0, _ = z.zeta_charpoly(ctx, s, policy="cover")
            P1, _ = z.zeta_charpoly(ctx, s, policy="learned", weights=w, hidden=8)
            assert P0 == P1
    finally:
        z.zeta_destroy(ctx)


@pytest.mark.gpu
def test_learned_policy_on_the_gpu_equals_the_oracle():
    # quintic curves over F_41 and F_47 (the largest moduli of the workload: 41^11 = 2^58.9) and F_7
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2602_24155_gb300.policy_train import train_policy
    ctx = z.zeta_create(0)
    try:
        w, _, _ = train_policy(ctx, [_instance("quintic_curves", i) for i in range(100, 124)], hidden=8, epochs=20)
        specs = [_instance("quintic_curves", i) for i in (9, 11, 12)]
        assert sorted(s[2] for s in specs) == [7, 41, 47]
        P, per, _ = z.zeta_batch(ctx, specs, policy="learned", weights=w, hidden=8)
        for s, Pi, st in zip(specs, P, per):
            ref = ozeta.compute_zeta(*s, policy="p_chunk")
            assert st["status"] == 0 and Pi == ref.P, s[2]
            F, Y, _ = z.zeta_frobenius(ctx, s, policy="learned", weights=w, hidden=8)
            assert (Y.astype(object) == ref.Y).all()
    finally:
        z.zeta_destroy(ctx)
