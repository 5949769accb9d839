"""Pins of the FP64 proposal / sparse-HAP reference: library kNN, finite-
difference gradients, special cases of candidate selection, and the masked
(-inf) similarity reading of sparse HAP."""
import numpy as np

from oracle import hap_oracle as H
from oracle import proposal_oracle as P
from paper_1403_7394_gb300 import workloads as W


def test_knn_matches_scipy():
    from scipy.spatial import cKDTree
    X, _ = W.gmm_points(300, 5, 6, sigma=1.0, seed=1)
    idx, dist = P.knn(X, 12)
    d, j = cKDTree(X).query(X, k=13)
    np.testing.assert_allclose(dist, d[:, 1:] ** 2, rtol=1e-12)
    np.testing.assert_array_equal(idx, j[:, 1:])


def test_mlp_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    Pm = P.mlp_init(6, 9, seed=3)
    Pm["b1"] = rng.normal(0, 0.1, 9)
    Pm["b2"] = rng.normal(0, 0.1, 9)
    F = rng.normal(size=(40, 6))
    y = (rng.random(40) < 0.3).astype(float)
    loss, G = P.bce_loss_and_grads(Pm, F, y, pos_weight=2.5)
    h = 1e-6
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        flat = Pm[name].reshape(-1)
        num = np.empty(flat.size)
        for q in range(flat.size):
            old = flat[q]
            flat[q] = old + h
            lp, _ = P.bce_loss_and_grads(Pm, F, y, 2.5)
            flat[q] = old - h
            lm, _ = P.bce_loss_and_grads(Pm, F, y, 2.5)
            flat[q] = old
            num[q] = (lp - lm) / (2 * h)
        np.testing.assert_allclose(np.asarray(G[name]).reshape(-1), num, rtol=1e-5, atol=1e-9, err_msg=name)


def test_mlp_forward_closed_form():
    """A network whose hidden layers copy (ReLU of) the inputs computes
    sum(relu(f)) + 1."""
    Pm = {"W1": np.eye(3), "b1": np.zeros(3), "W2": np.eye(3), "b2": np.zeros(3),
          "W3": np.ones(3), "b3": np.asarray(1.0)}
    F = np.array([[1.0, -2.0, 3.0], [-1.0, -1.0, 0.5]])
    z, _ = P.mlp_forward(Pm, F)
    np.testing.assert_allclose(z, [5.0, 1.5])


def test_candidates_special_cases():
    X, _ = W.gmm_points(50, 2, 3, sigma=0.8, seed=2)
    idx, _ = P.knn(X, 20)
    plain = P.select_candidates(idx, 8, 7)
    same = P.select_candidates(idx, 8, 7, score=np.zeros(50))
    np.testing.assert_array_equal(plain, same)  # K_near = K - 1: the scores pick nothing
    for i in range(50):
        assert i in plain[i] and np.all(np.diff(plain[i]) > 0)
    # a score that favours point 0 brings it into every pool that contains it
    score = np.zeros(50)
    score[0] = 10.0
    c = P.select_candidates(idx, 8, 4, score=score)
    for i in range(50):
        if 0 in idx[i, 4:]:
            assert 0 in c[i]


def test_full_candidate_graph_is_dense_hap_and_masked_hap_is_finite():
    X, _ = W.gmm_points(40, 2, 4, sigma=0.6, seed=5)
    S0 = H.neg_sq_euclidean(X)
    S = H.level_similarities(S0, [H.median_preference(S0)] * 2)
    cand_all = np.tile(np.arange(40, dtype=np.int32), (40, 1))
    Sm = np.stack([P.masked_similarity(S[l], cand_all) for l in range(2)])
    a, b = H.run(S, 10, 0.5, H.PAPER), H.run(Sm, 10, 0.5, H.PAPER)
    np.testing.assert_array_equal(a.A, b.A)
    np.testing.assert_array_equal(a.R, b.R)
    idx, _ = P.knn(X, 10)
    cand = P.select_candidates(idx, 6, 5)
    Sm = np.stack([P.masked_similarity(S[l], cand) for l in range(2)])
    st = H.run(Sm, 15, 0.5, H.PAPER)
    inside = np.zeros((40, 40), dtype=bool)
    inside[np.repeat(np.arange(40), 6), cand.reshape(-1)] = True
    for l in range(2):
        assert np.all(np.isfinite(st.R[l][inside])) and np.all(np.isneginf(st.R[l][~inside]))
        assert np.all(np.isfinite(st.A[l]))
    e = H.exemplars(st.A, st.R)
    assert np.all(inside[np.arange(40), e[0]])  # exemplars are always candidates


def test_hub_helpers():
    X, _ = W.gmm_points(120, 3, 4, sigma=0.8, seed=6)
    score = np.random.default_rng(2).normal(size=120)
    score[5] = score[7]  # a tie: lower index first
    hubs = P.top_scores(score, 12)
    assert list(hubs) == sorted(range(120), key=lambda i: (-score[i], i))[:12]
    hubnn, hd = P.knn_subset(X, hubs, 5)
    for i in range(120):
        d = {h: ((X[i] - X[h]) ** 2).sum() for h in hubs if h != i}
        best = sorted(d, key=lambda h: (d[h], h))[:5]
        assert list(hubnn[i]) == best
    pool, _ = P.knn(X, 10)
    c = P.select_hub_candidates(pool, hubnn, 8, 3)
    for i in range(120):
        assert i in c[i] and np.all(np.diff(c[i]) > 0)
        assert set(pool[i, :3]) <= set(c[i])
        assert hubnn[i, 0] in c[i]
