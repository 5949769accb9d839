"""Learned candidate proposal (kNN, features, MLP forward / gradients /
training, candidate selection) and sparse HAP on GB300 against the FP64
reference.  Sparse HAP is checked against dense HAP on a similarity that is
-inf outside the candidate graph."""
import numpy as np
import pytest
import torch

from oracle import hap_oracle as H
from oracle import proposal_oracle as P
from paper_1403_7394_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def hapm():
    from paper_1403_7394_gb300 import hap
    return hap


def _bf16(x):
    return torch.from_numpy(np.asarray(x, dtype=np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def _params_from_flat(theta, F, H_=128, round_weights=True):
    th = np.asarray(theta, dtype=np.float64)
    o = 0
    out = {}
    for name, shape in (("W1", (F, H_)), ("b1", (H_,)), ("W2", (H_, H_)), ("b2", (H_,)), ("W3", (H_,)), ("b3", ())):
        n = int(np.prod(shape)) if shape else 1
        v = th[o:o + n].reshape(shape) if shape else np.asarray(th[o])
        out[name] = _bf16(v) if (round_weights and name.startswith("W")) else v
        o += n
    return out


@pytest.mark.parametrize("N,d,M", [(1500, 32, 64), (700, 5, 100), (300, 2, 16)])
def test_knn_exact(N, d, M):
    hap = hapm()
    X, _ = W.gmm_points(N, d, 8, sigma=1.0, seed=d, means="normal", mean_scale=2.0)
    X32 = X.astype(np.float32)
    idx, dist = hap.knn(torch.from_numpy(X32).to(DEV), M)
    idx, dist = idx.cpu().numpy(), dist.cpu().numpy().astype(np.float64)
    ridx, rdist = P.knn(X32, M)
    assert np.abs(dist - rdist).max() <= 1e-5 * np.abs(rdist).max()
    # indices agree except where FP32 rounding reorders near-equal distances
    for i in np.nonzero(np.any(idx != ridx, axis=1))[0]:
        diff = set(idx[i]) ^ set(ridx[i])
        kth = rdist[i, -1]
        for j in diff:
            dj = ((X32[i].astype(np.float64) - X32[j]) ** 2).sum()
            assert abs(dj - kth) <= 1e-5 * kth, (i, j)
        assert np.all(np.diff(dist[i]) >= 0)


def test_features_match_reference():
    hap = hapm()
    X, _ = W.gmm_points(900, 16, 6, sigma=1.0, seed=1, means="normal", mean_scale=2.0)
    idx, dist = hap.knn(torch.from_numpy(X.astype(np.float32)).to(DEV), 32)
    feats, ls = hap.knn_features(dist, 16)
    d64 = dist.cpu().numpy().astype(np.float64)
    ref = P.knn_features(d64, 16, np.exp(np.mean(np.log(d64[:, 15]))))
    assert np.abs(feats.cpu().numpy() - ref).max() <= 1e-4


def test_mlp_forward_and_gradients_match_reference(report):
    hap = hapm()
    rng = np.random.default_rng(0)
    n, F = 2000, 16
    feats = rng.normal(size=(n, F)).astype(np.float32)
    labels = (rng.random(n) < 0.1).astype(np.float32)
    theta = hap.mlp_init_params(F, seed=5)
    theta[F * 128:F * 128 + 128] = rng.normal(0, 0.1, 128)  # nonzero biases
    mlp = hap.MLP(F, theta0=theta, device=DEV)
    ft = torch.from_numpy(feats).to(DEV)
    lt = torch.from_numpy(labels).to(DEV)
    Pm = _params_from_flat(theta, F)  # the BF16 weights the kernels use
    z_ref, _ = P.mlp_forward(Pm, feats.astype(np.float64))
    z = mlp.forward(ft).cpu().numpy()
    ez = np.abs(z - z_ref).max() / max(1.0, np.abs(z_ref).max())
    g, loss = mlp.gradients(ft, lt, pos_weight=9.0)
    loss_ref, G = P.bce_loss_and_grads(Pm, feats.astype(np.float64), labels, 9.0)
    gref = np.concatenate([np.asarray(G[k]).reshape(-1) for k in ("W1", "b1", "W2", "b2", "W3", "b3")])
    eg = np.abs(g - gref).max() / np.abs(gref).max()
    report(forward_err=float(ez), grad_err=float(eg), loss=loss, loss_ref=loss_ref)
    assert ez <= 1e-4
    assert abs(loss - loss_ref) <= 1e-5 * abs(loss_ref)
    assert eg <= 1e-4
    # Adam steps lower the loss
    l0 = mlp.train_step(ft, lt, 9.0, 3e-3, want_loss=True)
    for _ in range(150):
        last = mlp.train_step(ft, lt, 9.0, 3e-3, want_loss=True)
    assert last < 0.8 * l0


def test_candidate_selection_matches_reference():
    hap = hapm()
    X, _ = W.gmm_points(800, 8, 5, sigma=1.0, seed=2, means="normal", mean_scale=2.0)
    Xt = torch.from_numpy(X.astype(np.float32)).to(DEV)
    pool, _ = hap.knn(Xt, 64)
    score = torch.from_numpy(np.random.default_rng(1).normal(size=800).astype(np.float32)).to(DEV)
    for sc, kn in ((None, 31), (score, 12)):
        c = hap.select_candidates(pool, 32, kn, sc).cpu().numpy()
        ref = P.select_candidates(pool.cpu().numpy(), 32, kn, None if sc is None else sc.cpu().numpy())
        np.testing.assert_array_equal(c, ref)


def test_hub_selection_subset_knn_and_candidates():
    hap = hapm()
    N = 3000
    X, _ = W.gmm_points(N, 16, 12, sigma=1.0, seed=8, means="normal", mean_scale=2.0)
    X32 = X.astype(np.float32)
    Xt = torch.from_numpy(X32).to(DEV)
    score = np.random.default_rng(4).normal(size=N).astype(np.float32)
    score[10] = score[20]
    hubs = hap.top_scores(torch.from_numpy(score).to(DEV), 100).cpu().numpy()
    np.testing.assert_array_equal(hubs, P.top_scores(score, 100))
    hubnn, hd = hap.knn_subset(Xt, torch.from_numpy(hubs).to(DEV), 20)
    ridx, rd = P.knn_subset(X32, hubs, 20)
    assert np.abs(hd.cpu().numpy() - rd).max() <= 1e-5 * rd.max()
    mism = np.any(hubnn.cpu().numpy() != ridx, axis=1).mean()
    assert mism <= 0.01  # only FP32 near-ties may reorder
    pool, _ = hap.knn(Xt, 32)
    c = hap.select_hub_candidates(pool, hubnn, 40, 16).cpu().numpy()
    np.testing.assert_array_equal(c, P.select_hub_candidates(pool.cpu().numpy(), hubnn.cpu().numpy(), 40, 16))


def _sparse_problem(N, L, K, seed, K_near=None, score=None):
    hap = hapm()
    X, _ = W.gmm_points(N, 2, 6, sigma=0.6, seed=seed, means="uniform", mean_scale=10.0)
    X32 = X.astype(np.float32)
    Xt = torch.from_numpy(X32).to(DEV)
    pool, _ = hap.knn(Xt, min(100, N - 1))
    cand = hap.select_candidates(pool, K, K - 1 if K_near is None else K_near, score)
    S64 = H.neg_sq_euclidean(X32)
    p = H.median_preference(S64)
    prefs = np.array([p * (1 + 0.5 * l) for l in range(L)], dtype=np.float32)
    S_full = H.level_similarities(S64.astype(np.float32).astype(np.float64), prefs.astype(np.float64))
    cn = cand.cpu().numpy()
    S_mask = np.stack([P.masked_similarity(S_full[l], cn) for l in range(L)])
    return Xt, cand, cn, prefs, S_mask


@pytest.mark.parametrize("c_mode", ["paper", "fixed"])
def test_sparse_hap_equals_masked_dense_reference(c_mode, report):
    hap = hapm()
    N, L, K, T = 600, 3, 32, 4
    Xt, cand, cn, prefs, S_mask = _sparse_problem(N, L, K, seed=4)
    sp = hap.HAPSparse(N, L, K, prefs=prefs, damping=0.5, c_mode=c_mode, device=DEV)
    sp.set_candidates(cand, Xt)
    sp.iterate(T)
    g = sp.get_state()
    ref = H.run(S_mask, T, 0.5, c_mode)
    rows = np.repeat(np.arange(N), K)
    errs = {}
    for k in ("A", "R"):
        got = g[k].cpu().numpy().astype(np.float64)
        want = getattr(ref, k)[:, rows, cn.reshape(-1)].reshape(L, N, K)
        errs[k] = H.message_rel_error(got, want)
    for k in ("c", "tau", "phi"):
        errs[k] = H.message_rel_error(g[k].cpu().numpy().astype(np.float64), getattr(ref, k))
    e = sp.exemplars().cpu().numpy()
    report(errs=errs)
    assert all(v <= 1e-4 for v in errs.values()), errs
    np.testing.assert_array_equal(e, H.exemplars(ref.A, ref.R))


def test_full_candidate_graph_equals_dense_gpu():
    hap = hapm()
    N, L = 64, 2
    X, _ = W.gmm_points(N, 3, 3, sigma=0.7, seed=9)
    X32 = X.astype(np.float32)
    Xt = torch.from_numpy(X32).to(DEV)
    cand = torch.from_numpy(np.tile(np.arange(N, dtype=np.int32), (N, 1))).to(DEV)
    prefs = np.array([-6.0, -9.0], dtype=np.float32)
    sp = hap.HAPSparse(N, L, N, prefs=prefs, device=DEV)
    sp.set_candidates(cand, Xt)
    ctx = hap.HAP(N, L, prefs=prefs, device=DEV)
    ctx.build_similarity(Xt, mode="f32")
    sp.iterate(8)
    ctx.iterate(8)
    gs, gd = sp.get_state(), ctx.get_state()
    for k in ("A", "R", "c", "tau", "phi"):
        assert H.message_rel_error(gs[k].cpu().numpy(), gd[k].cpu().numpy()) <= 1e-5, k
    np.testing.assert_array_equal(sp.exemplars().cpu().numpy(), ctx.exemplars().cpu().numpy())
