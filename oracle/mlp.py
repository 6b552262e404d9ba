"""Float64 reference of the direction-scoring network (test infrastructure only).

Same architecture and parameter layout as the library's learned policy:
score = w3 . relu(W2^T relu(W1^T x + b1) + b2) + b3; a decision is a group of
rows; loss = mean over groups of -log softmax(scores of the group)[label].
Written with numpy from the definitions (chain rule by hand); pinned against
finite differences in the tests.
"""
import numpy as np

F = 18


def unpack(params, H):
    p = np.asarray(params, dtype=np.float64)
    o = 0
    W1 = p[o:o + F * H].reshape(F, H); o += F * H
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def forward(params, H, X):
    W1, b1, W2, b2, w3, b3 = unpack(params, H)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1 + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2 + b2
    h2 = np.maximum(z2, 0.0)
    return h2 @ w3 + b3, (X, z1, h1, z2, h2)


def loss_and_grad(params, H, X, group_off, labels):
    W1, b1, W2, b2, w3, b3 = unpack(params, H)
    s, (X, z1, h1, z2, h2) = forward(params, H, X)
    G = len(labels)
    ds = np.zeros_like(s)
    loss = 0.0
    for g in range(G):
        a, b = int(group_off[g]), int(group_off[g + 1])
        sg = s[a:b]
        mx = sg.max()
        e = np.exp(sg - mx)
        sm = e / e.sum()
        loss += (np.log(e.sum()) + mx - sg[labels[g]]) / G
        d = sm.copy()
        d[labels[g]] -= 1.0
        ds[a:b] = d / G
    d2 = (z2 > 0) * np.outer(ds, w3)
    d1 = (z1 > 0) * (d2 @ W2.T)
    grads = [X.T @ d1, d1.sum(0), h1.T @ d2, d2.sum(0), h2.T @ ds, np.array([ds.sum()])]
    return loss, np.concatenate([g.ravel() for g in grads])
