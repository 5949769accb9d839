"""FP64 reference for the learned candidate proposal and sparse HAP.

TEST INFRASTRUCTURE ONLY (same rules as hap_oracle): used by tests/ and the
CPU legs of bench.py, never by the product path.

The paper's method (§2) is dense: every node may pick every other node as
exemplar.  Pruning each row to K candidate exemplars is an extension of this
repository; its exact meaning is HAP on a similarity matrix whose entries
outside the candidate graph are -inf (§2 allows similarities down to -inf:
such a pair can never be chosen, contributes max(0, rho) = 0 to every column
sum and never wins a row maximum).  ``masked_similarity`` builds that matrix
so the dense reference in hap_oracle is the sparse method's reference too.

Definitions of the proposal (the repository's, not the paper's):
  * k nearest neighbours by squared Euclidean distance, self excluded, ties
    broken by lower index;
  * features of point j: log(d_q(j) / scale) for its q = 1..F nearest
    neighbour distances d_q (squared), scale a global constant;
  * MLP: logits = W3 relu(W2 relu(W1 f + b1) + b2) + b3 (row-vector form
    below), trained with positive-weighted binary cross-entropy;
  * candidates of row i: i itself, its K_near nearest neighbours, and the
    K - 1 - K_near members of its M-neighbour pool beyond those with the
    highest scores (lower pool position first on ties); without scores, the
    K - 1 nearest neighbours.  Stored sorted by index.
"""
from __future__ import annotations

import numpy as np


def knn(X, k):
    """Exact k nearest neighbours (squared Euclidean), self excluded; returns
    (idx int32 (N, k), dist float64 (N, k)) sorted by (distance, index)."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    idx = np.empty((n, k), dtype=np.int32)
    dist = np.empty((n, k))
    cols = np.arange(n)
    for i in range(n):
        d = ((X - X[i]) ** 2).sum(axis=1)
        d[i] = np.inf
        order = np.lexsort((cols, d))[:k]
        idx[i] = order
        dist[i] = d[order]
    return idx, dist


def knn_features(dist, F, scale):
    """f_q(j) = log(d_q(j) / scale), q < F (squared distances)."""
    d = np.asarray(dist, dtype=np.float64)[:, :F]
    return np.log(np.maximum(d, 1e-30) / scale)


def mlp_init(in_dim, width, seed):
    """Parameters {W1 (in, w), b1 (w), W2 (w, w), b2 (w), W3 (w,), b3 ()}
    with uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases."""
    rng = np.random.default_rng(seed)
    a1, a2 = 1.0 / np.sqrt(in_dim), 1.0 / np.sqrt(width)
    return {"W1": rng.uniform(-a1, a1, (in_dim, width)), "b1": np.zeros(width),
            "W2": rng.uniform(-a2, a2, (width, width)), "b2": np.zeros(width),
            "W3": rng.uniform(-a2, a2, width), "b3": np.zeros(())}


def mlp_forward(P, F):
    """Returns logits (n,) and the activations needed by the backward pass."""
    F = np.asarray(F, dtype=np.float64)
    z1 = F @ P["W1"] + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"] + P["b2"]
    h2 = np.maximum(z2, 0.0)
    out = h2 @ P["W3"] + P["b3"]
    return out, (F, z1, h1, z2, h2)


def bce_loss_and_grads(P, F, y, pos_weight):
    """Mean positive-weighted BCE with logits and its exact gradients:
    loss = mean_s w_s [softplus(z_s) - y_s z_s], w_s = pos_weight if y_s else 1."""
    z, (X, z1, h1, z2, h2) = mlp_forward(P, F)
    y = np.asarray(y, dtype=np.float64)
    w = np.where(y > 0.5, pos_weight, 1.0)
    n = z.shape[0]
    loss = float(np.mean(w * (np.logaddexp(0.0, z) - y * z)))
    g = w * (1.0 / (1.0 + np.exp(-z)) - y) / n        # d loss / d z
    G = {"W3": h2.T @ g, "b3": np.asarray(g.sum())}
    d2 = np.outer(g, P["W3"]) * (z2 > 0)
    G["W2"] = h1.T @ d2
    G["b2"] = d2.sum(axis=0)
    d1 = (d2 @ P["W2"].T) * (z1 > 0)
    G["W1"] = X.T @ d1
    G["b1"] = d1.sum(axis=0)
    return loss, G


def select_candidates(pool_idx, K, K_near, score=None):
    """Candidate exemplars per row (see module docstring), sorted by index."""
    pool_idx = np.asarray(pool_idx)
    n, M = pool_idx.shape
    out = np.empty((n, K), dtype=np.int32)
    for i in range(n):
        if score is None:
            chosen = list(pool_idx[i, :K - 1])
        else:
            near = list(pool_idx[i, :K_near])
            rest = pool_idx[i, K_near:]
            s = np.asarray(score, dtype=np.float64)[rest]
            order = np.lexsort((np.arange(rest.size), -s))[:K - 1 - K_near]
            chosen = near + list(rest[order])
        out[i] = np.sort(np.array([i] + chosen, dtype=np.int32))
    return out


def knn_subset(X, subset, k):
    """The k nearest members of ``subset`` for every point (global indices),
    a point never taking itself; ties to the lower global index."""
    X = np.asarray(X, dtype=np.float64)
    subset = np.asarray(subset)
    n = X.shape[0]
    idx = np.empty((n, k), dtype=np.int32)
    dist = np.empty((n, k))
    for i in range(n):
        d = ((X[subset] - X[i]) ** 2).sum(axis=1)
        d[subset == i] = np.inf
        order = np.lexsort((subset, d))[:k]
        idx[i] = subset[order]
        dist[i] = d[order]
    return idx, dist


def top_scores(score, H):
    """Indices of the H highest scores, lower index first on ties."""
    score = np.asarray(score, dtype=np.float64)
    return np.lexsort((np.arange(score.size), -score))[:H].astype(np.int32)


def select_hub_candidates(pool, hubnn, K, K_near):
    """Candidates of row i: i, its K_near nearest, its nearest hubs not yet
    taken, then further pool entries, up to K; sorted by index."""
    n = pool.shape[0]
    out = np.empty((n, K), dtype=np.int32)
    for i in range(n):
        sel = [i]
        for src in (pool[i, :K_near], hubnn[i], pool[i, K_near:]):
            for v in src:
                if len(sel) == K:
                    break
                if v >= 0 and v not in sel:
                    sel.append(int(v))
        out[i] = np.sort(np.array(sel, dtype=np.int32))
    return out


def masked_similarity(S, cand):
    """S with -inf outside the candidate graph (each row keeps its candidate
    columns, including the diagonal)."""
    S = np.asarray(S, dtype=np.float64)
    M = np.full_like(S, -np.inf)
    rows = np.repeat(np.arange(S.shape[0]), cand.shape[1])
    cols = np.asarray(cand).reshape(-1)
    M[rows, cols] = S[rows, cols]
    return M
