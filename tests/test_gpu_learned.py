"""What the trained proposal network gains over plain kNN candidates, and
over hubs chosen without it (seeded random scores; a density score with no
learning, -log of the distance to the 16th nearest neighbour), at the same
K, hub count and number of nearest neighbours kept, averaged over three test
instances.

The network is trained on the GPU (hand-written forward/backward/Adam
kernels) on exemplar labels from dense HAP runs of two training instances,
then scores the points of a third instance; the N/64 highest-scoring points
become hubs, and every row keeps itself, its 8 nearest neighbours and its
nearest hubs (K = 16 candidates).  Sparse HAP on these learned candidates is
compared with sparse HAP on the 15 nearest neighbours,
both judged against dense HAP on the same instance (ARI of the level-1
assignments and net-similarity gap, NS from the points in FP64).

Setting: 8192 points in 32-D, 32 Gaussian components of about 256 points,
L = 3, c fixed (the undamped Eq. 2.6 feedback makes every point its own
exemplar here), lambda = 0.9, 400 iterations, preference 4x the median
similarity at level 1 (x8, x12 above) - a setting where dense HAP converges
(34 self-consistent exemplars, ARI 0.98 with the generating components)."""
import numpy as np
import pytest
import torch

from oracle import hap_oracle as H
from paper_1403_7394_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
N, D, L, T, LAM, K = 8192, 32, 3, 400, 0.9, 16


def _instance(seed):
    X, lab = W.gmm_points(N, D, N // 256, sigma=1.0, seed=seed, means="normal", mean_scale=2.0)
    X32 = X.astype(np.float32)
    i, j = W.sample_pairs(N, 1 << 16, seed=seed + 7)
    df = X32[i].astype(np.float64) - X32[j]
    p = np.float32(np.median(-np.einsum("kd,kd->k", df, df)))
    return X32, lab, np.array([4.0 * p * (1 + l) for l in range(L)], dtype=np.float32)


def _dense(hap, X32, prefs):
    ctx = hap.HAP(N, L, prefs=prefs, damping=LAM, device=DEV, c_mode="fixed")
    ctx.build_similarity(torch.from_numpy(X32).to(DEV), mode="bf16_split")
    ctx.iterate(T)
    e = ctx.exemplars().cpu().numpy()
    ctx.close()
    return e


def test_learned_candidates_beat_nearest_neighbours(report):
    from paper_1403_7394_gb300 import hap
    feats, labels = [], []
    for seed in (1, 2):
        X32, _, prefs = _instance(seed)
        e = _dense(hap, X32, prefs)
        y = np.zeros(N, np.float32)
        for l in range(L):
            y[np.unique(e[l])] = 1.0  # chosen as an exemplar at some level
        _, dist = hap.knn(torch.from_numpy(X32).to(DEV), 128)
        f, _ = hap.knn_features(dist, 16)
        feats.append(f)
        labels.append(torch.from_numpy(y).to(DEV))
    Fm, Y = torch.cat(feats), torch.cat(labels)
    posw = float((1 - Y.mean()) / Y.mean())
    mlp = hap.MLP(16, seed=0, device=DEV)
    l0 = mlp.train_step(Fm, Y, posw, 3e-3, want_loss=True)
    for _ in range(400):
        mlp.train_step(Fm, Y, posw, 3e-3)
    l1 = mlp.train_step(Fm, Y, posw, 3e-3, want_loss=True)

    res = {k: {"ari": [], "gap": [], "n_exemplars": []} for k in ("knn", "learned", "random_hubs", "density_hubs")}
    dense_ex = []
    for seed in (3, 4, 5):  # three test instances
        X32, _, prefs = _instance(seed)
        e_dense = _dense(hap, X32, prefs)
        dense_ex.append(int(len(np.unique(e_dense[0]))))
        Xt = torch.from_numpy(X32).to(DEV)
        pref_t = torch.from_numpy(np.repeat(prefs[:, None], N, axis=1)).to(DEV)
        ns_dense = hap.net_similarity_points(Xt, torch.from_numpy(e_dense).to(DEV), pref_t)
        pool, dist = hap.knn(Xt, 32)
        f, _ = hap.knn_features(dist, 16)
        scores = {"learned": mlp.forward(f),
                  "random_hubs": torch.rand(N, generator=torch.Generator(device=DEV).manual_seed(seed), device=DEV),
                  "density_hubs": -torch.log(dist[:, 15].clamp_min(1e-30))}
        for name in res:
            if name == "knn":
                cand = hap.select_candidates(pool, K, K - 1, None)
            else:
                hubs = hap.top_scores(scores[name].contiguous(), N // 64)
                hubnn, _ = hap.knn_subset(Xt, hubs, K)
                cand = hap.select_hub_candidates(pool, hubnn, K, K // 2)
            sp = hap.HAPSparse(N, L, K, prefs=prefs, damping=LAM, c_mode="fixed", device=DEV)
            sp.set_candidates(cand, Xt)
            sp.iterate(T)
            e = sp.exemplars().cpu().numpy()
            ns = sp.net_similarity()
            sp.close()
            res[name]["ari"].append(H.adjusted_rand_index(e[0], e_dense[0]))
            res[name]["gap"].append(float((ns_dense[0] - ns[0]) / abs(ns_dense[0])))
            res[name]["n_exemplars"].append(int(len(np.unique(e[0]))))
    mean = {k: {m: float(np.mean(v[m])) for m in ("ari", "gap")} for k, v in res.items()}
    report(loss=[l0, l1], dense_exemplars=dense_ex, mean=mean, **res)
    print({"loss": [l0, l1], "dense_exemplars": dense_ex, "mean": mean, **res})
    assert l1 < l0
    assert mean["learned"]["ari"] >= mean["knn"]["ari"] + 0.3
    assert mean["learned"]["gap"] < 0.25 * mean["knn"]["gap"]
    # the trained scores choose better hubs than chance (measured on GB300:
    # gap 0.056 vs 0.258, ARI 0.922 vs 0.865) ...
    assert mean["learned"]["gap"] < 0.5 * mean["random_hubs"]["gap"]
    assert mean["learned"]["ari"] >= mean["random_hubs"]["ari"] + 0.02
    # ... but not better than ranking by the 16th-neighbour distance alone
    # (gap 0.059, ARI 0.927): the network has learned a density score.  This
    # is reported (parity report and stdout), not asserted either way.
