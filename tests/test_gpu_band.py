"""Row bands (the row partition of §3) through the C ABI: several bands of one
problem stepped on one device, the exchange being every band's buffer placed
in one array in band order.

- one band holding every row gives the bits of hap_iterate (same kernels, same
  launch shape, same summation order);
- several uneven bands against the FP64 reference, free-running from
  Algorithm 1's start (tolerance 1e-4 in the message metric, as every parity
  test), and config 0 as specified (200 iterations, Eq. 2.6 as printed) with
  identical exemplars at every level;
- clusters of CTAs per row (rows wider than one CTA) against the unbanded
  context: only the grouping of the column sums differs, so 1e-5;
- the call order and the band boundaries are checked.
"""
import numpy as np
import pytest
import torch

from oracle import hap_oracle as H
from paper_1403_7394_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL = 1e-4


def _hap():
    from paper_1403_7394_gb300 import hap
    return hap


def _problem(N, L, seed, s_dtype="f32"):
    X, _ = W.gmm_points(N, 2, 6, sigma=0.6, seed=seed, means="uniform", mean_scale=10.0)
    S32 = H.neg_sq_euclidean(X).astype(np.float32)
    S_used = torch.from_numpy(S32).to(torch.bfloat16).float().numpy() if s_dtype == "bf16" else S32
    p = np.float32(H.median_preference(S32.astype(np.float64)))
    prefs = np.array([p * (1.0 + 0.5 * l) for l in range(L)], dtype=np.float32)
    return S32, prefs, H.level_similarities(S_used.astype(np.float64), prefs.astype(np.float64))


def _np(st):
    return {k: (v.cpu().numpy().astype(np.float64) if torch.is_tensor(v) else v) for k, v in st.items()
            if k != "per_band"}


def _errs(g, ref):
    return {f: H.message_rel_error(g[f], getattr(ref, f)) for f in ("A", "R", "c", "tau", "phi")}


@pytest.mark.parametrize("c_mode", ["paper", "fixed"])
def test_one_band_equals_the_context_bitwise(c_mode):
    hap = _hap()
    N, L, lam, T = 1000, 3, 0.5, 6
    S32, prefs, _ = _problem(N, L, seed=21)
    S = torch.from_numpy(S32).to(DEV)
    ctx = hap.HAP(N, L, prefs=prefs, damping=lam, device=DEV, c_mode=c_mode)
    ctx.set_similarity(S)
    ctx.iterate(T)
    grp = hap.BandGroup(N, L, [0, N], prefs=prefs, damping=lam, device=DEV, c_mode=c_mode)
    assert grp.bands[0].query(hap.Q_GRID_CLUSTERS) == ctx.query(hap.Q_GRID_CLUSTERS)
    grp.set_similarity(S)
    grp.iterate(T)
    a, b = _np(ctx.get_state()), _np(grp.get_state())
    for f in ("A", "R", "c", "tau", "phi"):
        np.testing.assert_array_equal(b[f], a[f], err_msg=f)
    assert np.array_equal(grp.exemplars().cpu().numpy(), ctx.exemplars().cpu().numpy())
    grp.close()
    ctx.close()


@pytest.mark.parametrize("c_mode,s_dtype", [("paper", "f32"), ("fixed", "f32"), ("paper", "bf16")])
def test_uneven_bands_against_the_reference(c_mode, s_dtype, report):
    hap = _hap()
    N, L, lam = 1300, 3, 0.6
    bounds = [0, 137, 640, 641, N]  # a one-row band and ragged band edges
    S32, prefs, S_ref = _problem(N, L, seed=22, s_dtype=s_dtype)
    grp = hap.BandGroup(N, L, bounds, prefs=prefs, damping=lam, device=DEV, c_mode=c_mode, s_dtype=s_dtype)
    grp.set_similarity(torch.from_numpy(S32).to(DEV))
    st = H.init_state(L, N)
    for t in range(1, 6):
        grp.iterate(1)
        st = H.step(S_ref, st, lam, c_mode)
        errs = _errs(_np(grp.get_state()), st)
        report(t=t, errs=errs)
        assert max(errs.values()) <= TOL, (t, errs)
    e_ref = H.exemplars(st.A, st.R)
    np.testing.assert_array_equal(grp.exemplars().cpu().numpy(), e_ref)
    grp.close()


def test_config0_in_four_bands_identical_exemplars(report):
    """Config 0 as specified (N = 500 points, L = 3, median preference,
    lambda = 0.5, 200 iterations, Eq. 2.6 as printed) in four row bands."""
    hap = _hap()
    N, L, lam, T = 500, 3, 0.5, 200
    X, _ = W.config0(seed=0)
    S32 = H.neg_sq_euclidean(X).astype(np.float32)
    p = np.float32(H.median_preference(S32.astype(np.float64)))
    prefs = np.full(L, p, dtype=np.float32)
    S_ref = H.level_similarities(S32.astype(np.float64), prefs.astype(np.float64))
    bounds = [0, 125, 250, 375, N]
    grp = hap.BandGroup(N, L, bounds, prefs=prefs, damping=lam, device=DEV)
    grp.set_similarity(torch.from_numpy(S32).to(DEV))
    grp.iterate(T)
    ref = H.run(S_ref, T, lam, H.PAPER, partition=[np.arange(bounds[r], bounds[r + 1]) for r in range(4)])
    e_ref = H.exemplars(ref.A, ref.R)
    e_gpu = grp.exemplars().cpu().numpy()
    errs = _errs(_np(grp.get_state()), ref)
    report(errs=errs, exemplars_equal=bool(np.array_equal(e_gpu, e_ref)))
    np.testing.assert_array_equal(e_gpu, e_ref)
    grp.close()


def test_clustered_rows_against_the_context(report):
    """Rows of 9000 columns take clusters of CTAs; two bands against the
    unbanded context (the column sums grouped differently: 1e-5)."""
    hap = _hap()
    N, L, lam, T = 9000, 2, 0.5, 3
    S32, prefs, _ = _problem(N, L, seed=23)
    S = torch.from_numpy(S32).to(DEV)
    ctx = hap.HAP(N, L, prefs=prefs, damping=lam, device=DEV)
    ctx.set_similarity(S)
    ctx.iterate(T)
    a = _np(ctx.get_state())
    ctx.close()
    grp = hap.BandGroup(N, L, [0, 4321, N], prefs=prefs, damping=lam, device=DEV)
    assert grp.bands[0].query(hap.Q_CLUSTER_SIZE) > 1
    grp.set_similarity(S)
    grp.iterate(T)
    b = _np(grp.get_state())
    errs = {f: H.message_rel_error(b[f], a[f]) for f in ("A", "R", "c", "tau", "phi")}
    report(errs=errs, cluster_size=grp.bands[0].query(hap.Q_CLUSTER_SIZE))
    assert max(errs.values()) <= 1e-5, errs
    grp.close()


def test_call_order_and_bounds_are_checked():
    hap = _hap()
    N, L = 300, 2
    S32, prefs, _ = _problem(N, L, seed=24)
    b = hap.HAPBand(N, 100, 100, L, prefs=prefs, device=DEV)
    b.set_similarity(torch.from_numpy(S32[100:200]).to(DEV))
    xall = torch.zeros((3, b.exchange_floats), dtype=torch.float32, device=DEV)
    with pytest.raises(hap.HapError) as e:
        b.columns(xall, [0, 100, 200, N])  # before the row pass
    assert e.value.code == hap.HAP_EINVAL
    b.rows(xall[1])
    with pytest.raises(hap.HapError) as e:
        b.rows(xall[1])  # twice in one iteration
    assert e.value.code == hap.HAP_EINVAL
    for bad in ([0, 100, 250, N], [0, 150, 200, N], [1, 100, 200, N], [0, 100, 200, N - 1]):
        with pytest.raises(hap.HapError) as e:
            b.columns(xall, bad)  # no band equal to this one, or not covering 0 .. N
        assert e.value.code == hap.HAP_EINVAL
    b.columns(xall, [0, 100, 200, N])
    b.sync()
    b.close()
    with pytest.raises(hap.HapError) as e:
        hap.HAPBand(N, 250, 100, L, device=DEV)  # past the last row
    assert e.value.code == hap.HAP_EINVAL
    with pytest.raises(hap.HapError) as e:
        hap.HAPBand(N, 0, 100, L, device=DEV, schedule="gauss_seidel")
    assert e.value.code == hap.HAP_EUNSUPPORTED
