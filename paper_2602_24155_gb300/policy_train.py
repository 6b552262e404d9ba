"""Training of the learned direction policy (ZETA_POLICY_LEARNED).

Decisions are generated by the library's own game (zeta_policy_dataset:
rollouts of the cover game label each sampled decision with its cheapest
direction) on a set of training instances, one host thread per instance,
concatenated in a seeded shuffled order of groups, and the network is trained
with the library's GPU kernels (zeta_mlp_train).
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import zeta_mlp_init, zeta_mlp_train, zeta_policy_dataset, POLICY_FEATURES


def build_dataset(specs, seed=0, opt=None):
    """opt: options of the instances' games (e.g. r=1 for a relative-precision-1 workload)."""
    Xs, offs, labs = [], [], []
    with ThreadPoolExecutor(max_workers=min(len(specs), os.cpu_count() or 1) or 1) as pool:
        sets = list(pool.map(lambda spec: zeta_policy_dataset(spec, **(opt or {})), specs))
    for X, go, lab, _ in sets:
        for g in range(len(lab)):
            Xs.append(X[go[g]:go[g + 1]])
            labs.append(int(lab[g]))
    order = np.random.default_rng(seed).permutation(len(labs))
    X = np.concatenate([Xs[g] for g in order]) if labs else np.zeros((0, POLICY_FEATURES), np.float32)
    sizes = np.array([len(Xs[g]) for g in order], dtype=np.uint32)
    go = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint32)
    lab = np.array([labs[g] for g in order], dtype=np.uint32)
    return X.astype(np.float32), go, lab


def train_policy(ctx, specs, hidden=64, epochs=30, batch_groups=512, lr=2e-3, seed=0, opt=None):
    """Returns (weights, final_loss, number of decisions)."""
    X, go, lab = build_dataset(specs, seed, opt)
    w = zeta_mlp_init(hidden, seed)
    w, loss = zeta_mlp_train(ctx, hidden, w, X, go, lab, epochs, batch_groups, lr)
    return w, loss, len(lab)
