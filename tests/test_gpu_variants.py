"""Method variants on the GPU against the FP64 reference (same tolerance and
error metric as test_gpu_parity): Algorithm 1's sequential level schedule,
Eq. 2.7 (kappa > 0), the paper's random per-point preferences, purity, and
the option combinations the library refuses."""
import numpy as np
import pytest
import torch

from oracle import hap_oracle as H
from paper_1403_7394_gb300 import workloads as W
from test_gpu_parity import DEV, assert_close, gpu_state, hap_mod, make_ctx, problem, to32

pytestmark = pytest.mark.gpu

GS_SHAPES = [
    (37, 3, {}),
    (1000, 4, {"col_sums": "tmem"}),
    (2051, 2, {"col_sums": "smem", "elems_per_thread": 8}),
    (3000, 3, {"cluster_size": 2, "col_sums": "tmem", "elems_per_thread": 8}),
]


@pytest.mark.parametrize("c_mode", ["paper", "fixed"])
@pytest.mark.parametrize("N,L,opt", GS_SHAPES, ids=[f"N{n}-L{l}" for n, l, _ in GS_SHAPES])
def test_gauss_seidel_teacher_forced(N, L, opt, c_mode, report):
    """One and two iterations of the sequential schedule from a reference
    state (c and phi carried in the state, reading R11)."""
    lam = 0.5
    S32, prefs, S_ref = problem(N, L, seed=N + 1)
    st = to32(H.run(S_ref, 3, lam, c_mode, schedule=H.GAUSS_SEIDEL))
    st.phi = st.phi.astype(np.float32).astype(np.float64)
    ctx = make_ctx(N, L, prefs, lam, S32, c_mode=c_mode, schedule="gauss_seidel", **opt)
    ctx.set_state(st.A, st.R, st.c, st.t, phi=st.phi)
    ctx.iterate(1)
    ref1 = H.step(S_ref, st, lam, c_mode, H.GAUSS_SEIDEL)
    e1 = assert_close(gpu_state(ctx), ref1)
    ctx.iterate(1)
    ref2 = H.step(S_ref, ref1, lam, c_mode, H.GAUSS_SEIDEL)
    e2 = assert_close(gpu_state(ctx), ref2)
    report(shape=ctx.shape, one_step=e1, two_steps=e2)
    ctx.close()


@pytest.mark.parametrize("s_dtype", ["f32", "bf16"])
def test_gauss_seidel_from_scratch(s_dtype, report):
    """Algorithm 1 literally: from its initial values, c and tau updated from
    the first iteration, 5 iterations free-running."""
    N, L, lam = 600, 3, 0.6
    S32, prefs, S_ref = problem(N, L, seed=21, s_dtype=s_dtype)
    ctx = make_ctx(N, L, prefs, lam, S32, s_dtype=s_dtype, schedule="gauss_seidel")
    st = H.init_state(L, N)
    for t in range(1, 6):
        ctx.iterate(1)
        st = H.step(S_ref, st, lam, H.PAPER, H.GAUSS_SEIDEL)
        report(t=t, errs=assert_close(gpu_state(ctx), st))
    e = ctx.exemplars().cpu().numpy()
    ref_e = H.exemplars(st.A, st.R)
    assert (e == ref_e).mean() > 0.99


@pytest.mark.parametrize("kappa", [0.25, 1.0])
@pytest.mark.parametrize("opt", [{}, {"col_sums": "smem", "elems_per_thread": 4, "cluster_size": 4}])
def test_similarity_level_update_teacher_forced(kappa, opt, report):
    """Eq. 2.7 (reading R10) inside the fused row pass: one and two
    iterations from a reference state."""
    N, L, lam = 1500, 3, 0.5
    S32, prefs, S_ref = problem(N, L, seed=33)
    st = to32(H.run(S_ref, 3, lam, H.PAPER, kappa=kappa))
    ctx = make_ctx(N, L, prefs, lam, S32, kappa=kappa, **opt)
    ctx.set_state(st.A, st.R, st.c, st.t)
    ctx.iterate(1)
    ref1 = H.step(S_ref, st, lam, H.PAPER, kappa=kappa)
    e1 = assert_close(gpu_state(ctx), ref1)
    ctx.iterate(1)
    ref2 = H.step(S_ref, ref1, lam, H.PAPER, kappa=kappa)
    e2 = assert_close(gpu_state(ctx), ref2)
    report(shape=ctx.shape, kappa=kappa, one_step=e1, two_steps=e2)
    ctx.close()


def test_similarity_level_update_from_scratch(report):
    N, L, lam, kappa = 700, 4, 0.5, 0.5
    S32, prefs, S_ref = problem(N, L, seed=34)
    ctx = make_ctx(N, L, prefs, lam, S32, kappa=kappa, c_mode="fixed")
    st = H.init_state(L, N)
    for t in range(1, 5):
        ctx.iterate(1)
        st = H.step(S_ref, st, lam, H.FIXED, kappa=kappa)
        report(t=t, errs=assert_close(gpu_state(ctx), st))


def test_random_point_preferences_image_like(report):
    """§4.1's image set-up on a synthetic stand-in: RGB pixels of a 40 x 40
    procedural image (0..255), S = -squared distance, a preference per point
    and level drawn uniformly in [-1e6, 0], L = 3, lambda = 0.5, 30
    iterations; teacher-forced parity at t = 30 and free-running exemplars."""
    hap = hap_mod()
    rng = np.random.default_rng(5)
    h = w = 40
    yy, xx = np.mgrid[0:h, 0:w]
    regions = (xx // 14) + 3 * (yy // 14)
    palette = rng.uniform(0, 255, size=(9, 3))
    img = np.clip(palette[regions] + rng.normal(0, 6.0, size=(h, w, 3)), 0, 255)
    X = img.reshape(-1, 3)
    N, L, lam = X.shape[0], 3, 0.5
    S32 = H.neg_sq_euclidean(X).astype(np.float32)
    P = rng.uniform(-1e6, 0.0, size=(L, N)).astype(np.float32)
    S_ref = np.repeat(S32.astype(np.float64)[None], L, axis=0)
    for l in range(L):
        np.fill_diagonal(S_ref[l], P[l])
    ctx = hap.HAP(N, L, damping=lam, device=DEV)
    ctx.set_preferences(P)
    ctx.set_similarity(torch.from_numpy(S32).to(DEV))
    ctx.iterate(29)
    g = gpu_state(ctx)
    st = H.HAPState(g["A"], g["R"], g["c"], g["tau"], g["phi"], 29)
    ctx.iterate(1)
    errs = assert_close(gpu_state(ctx), H.step(S_ref, st, lam, H.PAPER))
    ref = H.run(S_ref, 30, lam, H.PAPER)
    e_gpu = ctx.exemplars().cpu().numpy()
    e_ref = H.exemplars(ref.A, ref.R)
    labels = H.hierarchical_labels(e_ref)
    report(errs=errs, exemplar_match=float((e_gpu == e_ref).mean()),
           purity_level1=H.purity(labels[0], regions.ravel()))
    assert (e_gpu[0] == e_ref[0]).mean() > 0.99


def test_purity_of_gpu_clustering(report):
    """Purity (§4) of the GPU's level-1 clusters on a well-separated mixture
    equals the reference's (same exemplars) and is high."""
    N, L, lam = 800, 2, 0.9
    X, truth = W.gmm_points(N, 2, 8, sigma=0.4, seed=12, means="uniform", mean_scale=12.0)
    S32 = H.neg_sq_euclidean(X).astype(np.float32)
    p = np.float32(H.median_preference(S32.astype(np.float64)))
    prefs = np.array([p, 4 * p], dtype=np.float32)
    S_ref = H.level_similarities(S32.astype(np.float64), prefs.astype(np.float64))
    ctx = make_ctx(N, L, prefs, lam, S32, c_mode="fixed")
    ctx.iterate(200)
    e_gpu = ctx.exemplars().cpu().numpy()
    ref = H.run(S_ref, 200, lam, H.FIXED)
    e_ref = H.exemplars(ref.A, ref.R)
    pg = H.purity(H.hierarchical_labels(e_gpu)[0], truth)
    pr = H.purity(H.hierarchical_labels(e_ref)[0], truth)
    report(purity_gpu=pg, purity_ref=pr)
    assert pg == pr and pg > 0.9


def test_variant_options_refused():
    hap = hap_mod()
    for opt in ({"schedule": "gauss_seidel", "kappa": 0.5}, {"kappa": 0.5, "s_per_level": True}):
        with pytest.raises(hap.HapError) as ei:
            hap.HAP(64, 2, device=DEV, **opt)
        assert ei.value.code == hap.HAP_EUNSUPPORTED
    for k in (-0.1, 1.5, float("nan")):
        with pytest.raises(hap.HapError) as ei:
            hap.HAP(64, 2, device=DEV, kappa=k)
        assert ei.value.code == hap.HAP_EINVAL
    with pytest.raises(hap.HapError) as ei:
        hap.HAPBatch([64, 100], [2, 3], device=DEV, schedule="gauss_seidel")
    assert ei.value.code == hap.HAP_EUNSUPPORTED


def test_gauss_seidel_per_level_asymmetric_similarity(report):
    """The sequential schedule with a separate non-metric S per level (§2)."""
    hap = hap_mod()
    N, L, lam = 500, 3, 0.5
    mats = [problem(N, 1, seed=60 + l, asym=True)[0] for l in range(L)]
    prefs = np.array([-30.0, -60.0, -90.0], dtype=np.float32)
    S_ref = np.stack([m.astype(np.float64) for m in mats])
    for l in range(L):
        np.fill_diagonal(S_ref[l], prefs[l])
    ctx = hap.HAP(N, L, prefs=prefs, damping=lam, device=DEV, s_per_level=True, schedule="gauss_seidel")
    for l in range(L):
        ctx.set_similarity(torch.from_numpy(mats[l]).to(DEV), level=l)
    st = to32(H.run(S_ref, 3, lam, H.PAPER, schedule=H.GAUSS_SEIDEL))
    st.phi = st.phi.astype(np.float32).astype(np.float64)
    ctx.set_state(st.A, st.R, st.c, st.t, phi=st.phi)
    ctx.iterate(2)
    ref = H.step(S_ref, H.step(S_ref, st, lam, H.PAPER, H.GAUSS_SEIDEL), lam, H.PAPER, H.GAUSS_SEIDEL)
    report(errs=assert_close(gpu_state(ctx), ref))


def test_similarity_level_update_bf16_storage(report):
    """Eq. 2.7 on a BF16-stored S (the chain runs in FP32 registers)."""
    N, L, lam, kappa = 900, 3, 0.5, 0.5
    S32, prefs, S_ref = problem(N, L, seed=35, s_dtype="bf16")
    st = to32(H.run(S_ref, 3, lam, H.FIXED, kappa=kappa))
    ctx = make_ctx(N, L, prefs, lam, S32, kappa=kappa, c_mode="fixed", s_dtype="bf16")
    ctx.set_state(st.A, st.R, st.c, st.t)
    ctx.iterate(2)
    ref = H.step(S_ref, H.step(S_ref, st, lam, H.FIXED, kappa=kappa), lam, H.FIXED, kappa=kappa)
    report(errs=assert_close(gpu_state(ctx), ref))
