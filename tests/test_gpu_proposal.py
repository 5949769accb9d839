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


@pytest.mark.parametrize("method", ["cuda_cores", "tensor_cores"])
@pytest.mark.parametrize("N,d,M", [(1500, 32, 64), (700, 5, 100), (300, 2, 16), (2100, 64, 64)])
def test_knn_exact(N, d, M, method):
    hap = hapm()
    if method == "tensor_cores" and M > 64:
        pytest.skip("the tensor-core first pass keeps at most 80 candidates (M <= 64)")
    X, _ = W.gmm_points(N, d, 8, sigma=1.0, seed=d, means="normal", mean_scale=2.0)
    X32 = X.astype(np.float32)
    idx, dist = hap.knn(torch.from_numpy(X32).to(DEV), M, method=method)
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


def test_knn_tensor_cores_match_cuda_cores(report):
    """At a size where the tensor-core path is the automatic choice (and the
    points are first sorted by nearest pivot), its re-ranked result equals
    the CUDA-core kNN (same FP32 distance arithmetic) row for row; hub kNN (a
    subset of candidates) likewise up to the order of exactly equal
    distances."""
    hap = hapm()
    X, _ = W.gmm_points(20000, 32, 64, sigma=1.0, seed=8, means="normal", mean_scale=2.0)
    Xt = torch.from_numpy(X.astype(np.float32)).to(DEV)
    i_tc, d_tc = hap.knn(Xt, 32, method="tensor_cores")
    i_cc, d_cc = hap.knn(Xt, 32, method="cuda_cores")
    same = (i_tc == i_cc).all(dim=1).float().mean().item()
    report(rows_identical=same)
    assert same == 1.0 and torch.equal(d_tc, d_cc)
    # subsets of several sizes (queries never take their own point)
    for ns in (700, 2500, 5000):
        sub = torch.from_numpy(np.sort(np.random.default_rng(1).choice(20000, ns, replace=False)).astype(np.int32)).to(DEV)
        s_tc, e_tc = hap.knn_subset(Xt, sub, 48, method="tensor_cores")
        s_cc, e_cc = hap.knn_subset(Xt, sub, 48, method="cuda_cores")
        assert torch.equal(e_tc, e_cc), ns
        assert torch.equal(torch.sort(s_tc, dim=1).values, torch.sort(s_cc, dim=1).values), ns


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


def test_exemplar_points_and_refined_candidates():
    """hap_exemplar_points lists the distinct valid exemplar indices in
    increasing order (np.unique); the refined candidates are the hub
    candidates with exactly those points as hubs, also when there are fewer
    exemplars than K."""
    hap = hapm()
    N, K, K_near = 2000, 32, 4
    rng = np.random.default_rng(9)
    e = rng.integers(-3, N + 3, size=(3, N)).astype(np.int32)  # entries outside [0, N) are ignored
    e[:, ::7] = 5
    pts = hap.exemplar_points(torch.from_numpy(e).to(DEV), N).cpu().numpy()
    np.testing.assert_array_equal(pts, np.unique(e[(e >= 0) & (e < N)]))
    X, _ = W.gmm_points(N, 8, 10, sigma=1.0, seed=12, means="normal", mean_scale=2.0)
    X32 = X.astype(np.float32)
    Xt = torch.from_numpy(X32).to(DEV)
    pool, _ = hap.knn(Xt, 16)
    for n_ex in (20, 300):  # fewer and more exemplars than K
        ex = np.sort(rng.choice(N, n_ex, replace=False)).astype(np.int32)
        e2 = ex[rng.integers(0, n_ex, size=(2, N))]
        e2[0, :n_ex] = ex  # every one of them used
        cand = hap.refine_candidates(Xt, pool, torch.from_numpy(e2).to(DEV), K, K_near).cpu().numpy()
        hubnn, _ = hap.knn_subset(Xt, torch.from_numpy(ex).to(DEV), min(K, n_ex))
        want = P.select_hub_candidates(pool.cpu().numpy(), hubnn.cpu().numpy(), K, K_near)
        np.testing.assert_array_equal(cand, want)
        ridx, _ = P.knn_subset(X32, ex, min(K, n_ex))
        assert np.any(hubnn.cpu().numpy() != ridx, axis=1).mean() <= 0.01  # FP32 near-ties only


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
@pytest.mark.parametrize("N,K,L", [(600, 32, 3), (602, 30, 3), (601, 31, 6), (700, 64, 3), (701, 64, 1),
                                   (703, 64, 2), (700, 64, 4), (705, 64, 5)])
def test_sparse_hap_equals_masked_dense_reference(c_mode, N, K, L, report):
    """Even and odd row and candidate counts; L = 6 takes the column terms b
    of levels 4 and 5 from a second 16-byte gather per candidate; K = 64 runs
    the variant where every lane holds two entries (L = 1 to 4), and with
    L = 5 the variant with a second gather of b."""
    hap = hapm()
    T = 4
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


@pytest.mark.parametrize("K,L", [(48, 2), (64, 3)])
def test_sparse_hub_columns_against_reference(K, L, report):
    """A candidate graph with hub columns (every row keeps itself, its 20
    nearest neighbours and shared hubs out of 40, so hub columns hold about
    2000-3000 entries) and N > 512 (two radix passes in the GPU column index):
    sparse HAP against the dense reference on the masked similarity, and
    bitwise repeatable."""
    hap = hapm()
    N, T = 3000, 3
    X, _ = W.gmm_points(N, 3, 8, sigma=0.7, seed=21, means="uniform", mean_scale=10.0)
    X32 = X.astype(np.float32)
    nn, _ = P.knn(X32, 20)
    rng = np.random.default_rng(3)
    hubs = rng.choice(N, 40, replace=False)
    cn = np.empty((N, K), np.int32)
    for i in range(N):
        sel = [i] + [int(v) for v in nn[i]]
        for hb in rng.permutation(hubs):
            if len(sel) == K:
                break
            if hb not in sel:
                sel.append(int(hb))
        extra = 0
        while len(sel) < K:  # rows whose neighbours overlap the hubs
            if extra not in sel:
                sel.append(extra)
            extra += 1
        cn[i] = np.sort(sel)
    S64 = H.neg_sq_euclidean(X32.astype(np.float64))
    prefs = np.array([-60.0, -120.0, -180.0][:L], dtype=np.float32)
    S_full = H.level_similarities(S64, prefs.astype(np.float64))
    S_mask = np.stack([P.masked_similarity(S_full[l], cn) for l in range(L)])
    Xt = torch.from_numpy(X32).to(DEV)
    cand = torch.from_numpy(cn).to(DEV)
    outs = []
    for _ in range(2):
        sp = hap.HAPSparse(N, L, K, prefs=prefs, damping=0.5, c_mode="paper", device=DEV)
        sp.set_candidates(cand, Xt)
        sp.iterate(T)
        outs.append(sp.get_state())
        sp.close()
    for k in ("A", "R", "c", "tau", "phi"):
        assert torch.equal(outs[0][k], outs[1][k]), k
    # the GPU's s uses the points' FP32 direct differences; the reference's S
    # comes from the same FP32 points in FP64
    ref = H.run(S_mask, T, 0.5, H.PAPER)
    rows = np.repeat(np.arange(N), K)
    errs = {}
    for k in ("A", "R"):
        got = outs[0][k].cpu().numpy().astype(np.float64)
        errs[k] = H.message_rel_error(got, getattr(ref, k)[:, rows, cn.reshape(-1)].reshape(L, N, K))
    for k in ("c", "tau", "phi"):
        errs[k] = H.message_rel_error(outs[0][k].cpu().numpy().astype(np.float64), getattr(ref, k))
    report(errs=errs, max_column=int(np.bincount(cn.reshape(-1)).max()))
    assert all(v <= 1e-4 for v in errs.values()), errs


def test_net_similarity_points_matches_fp64():
    """NS^l = sum_i -||x_i - x_{e_i}||^2 (preference where e_i = i) from the
    points, in FP64 on the GPU (chunked, fixed order), against numpy FP64;
    N not a multiple of the chunk count, exemplars mixing self and others."""
    hap = hapm()
    rng = np.random.default_rng(12)
    N, d, L = 5003, 7, 3
    X32 = rng.normal(size=(N, d)).astype(np.float32)
    e = rng.integers(0, N, size=(L, N)).astype(np.int32)
    e[:, ::5] = np.arange(N, dtype=np.int32)[::5]
    pref = (-rng.uniform(1, 5, size=(L, N))).astype(np.float32)
    got = hap.net_similarity_points(torch.from_numpy(X32).to(DEV), torch.from_numpy(e).to(DEV),
                                    torch.from_numpy(pref).to(DEV))
    X64 = X32.astype(np.float64)
    want = np.empty(L)
    for l in range(L):
        dd = ((X64 - X64[e[l]]) ** 2).sum(axis=1)
        self_ = e[l] == np.arange(N)
        want[l] = np.where(self_, pref[l].astype(np.float64), -dd).sum()
    np.testing.assert_allclose(got, want, rtol=1e-12)


def test_sparse_candidates_rejected():
    hap = hapm()
    N, K = 50, 4
    Xt = torch.zeros((N, 2), device=DEV)
    good = np.stack([np.sort(np.array([i, (i + 1) % N, (i + 2) % N, (i + 3) % N])) for i in range(N)]).astype(np.int32)
    sp = hap.HAPSparse(N, 1, K, device=DEV)
    sp.set_candidates(torch.from_numpy(good).to(DEV), Xt)
    for bad in (good[:, ::-1].copy(),                                   # not increasing
                np.where(good == np.arange(N)[:, None], (np.arange(N)[:, None] + 10) % N, good),  # no self
                np.where(good == 3, N + 7, good)):                      # out of range
        with pytest.raises(hap.HapError) as ei:
            sp.set_candidates(torch.from_numpy(np.ascontiguousarray(bad, dtype=np.int32)).to(DEV), Xt)
        assert ei.value.code == hap.HAP_EINVAL
    sp.set_candidates(torch.from_numpy(good).to(DEV), Xt)
    sp.iterate(2)
    sp.close()
