"""Batched instances (one persistent launch per iteration) against the
single-instance path and the FP64 reference."""
import numpy as np
import pytest
import torch

from oracle import hap_oracle as H
from paper_1403_7394_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = 1e-4


def _instances(Ns, Ls, seed=0, d=2):
    out = []
    for q, (n, l) in enumerate(zip(Ns, Ls)):
        X, _ = W.gmm_points(n, d, 5, sigma=0.6, seed=seed + q, means="uniform", mean_scale=10.0)
        S32 = H.neg_sq_euclidean(X).astype(np.float32)
        p = np.float32(H.median_preference(S32.astype(np.float64)))
        prefs = np.array([p * (1.0 + 0.5 * k) for k in range(l)], dtype=np.float32)
        out.append((X.astype(np.float32), S32, prefs))
    return out


def _np(x):
    return x.cpu().numpy().astype(np.float64) if torch.is_tensor(x) else np.asarray(x, dtype=np.float64)


def _errs(g, ref):
    get = (lambda k: ref[k]) if isinstance(ref, dict) else (lambda k: getattr(ref, k))
    return {k: H.message_rel_error(_np(g[k]), _np(get(k))) for k in ("A", "R", "c", "tau", "phi")}


@pytest.mark.parametrize("c_mode", ["paper", "fixed"])
def test_batch_matches_single_instances(c_mode, report):
    from paper_1403_7394_gb300 import hap
    Ns = [37, 200, 513, 1000, 2100, 4000, 256, 97]
    Ls = [2, 3, 1, 4, 2, 3, 4, 1]
    insts = _instances(Ns, Ls, seed=100)
    bt = hap.HAPBatch(Ns, Ls, damping=0.5, device=DEV, c_mode=c_mode)
    bt.set_preferences([x[2] for x in insts])
    for b, (_, S32, _) in enumerate(insts):
        bt.set_similarity(b, torch.from_numpy(S32).to(DEV))
    T = 6  # iteration 1 direct, then graph replays
    bt.iterate(T)
    e_b = [x.cpu().numpy() for x in bt.exemplars()]
    ns_b = bt.net_similarity()
    worst = 0.0
    for b, (_, S32, prefs) in enumerate(insts):
        ctx = hap.HAP(Ns[b], Ls[b], prefs=prefs, damping=0.5, device=DEV, c_mode=c_mode)
        ctx.set_similarity(torch.from_numpy(S32).to(DEV))
        ctx.iterate(T)
        errs = _errs(bt.get_state(b), ctx.get_state())
        worst = max(worst, max(errs.values()))
        assert all(e <= TOL for e in errs.values()), (b, errs)
        np.testing.assert_array_equal(e_b[b], ctx.exemplars().cpu().numpy())
        np.testing.assert_allclose(ns_b[b], ctx.net_similarity(), rtol=1e-9)
        ctx.close()
    report(worst=worst, launches=bt.query(7))
    bt.close()


def test_batch_against_reference_and_tuner():
    from paper_1403_7394_gb300 import hap
    Ns, Ls = [300, 64, 700], [3, 2, 2]
    insts = _instances(Ns, Ls, seed=7)
    bt = hap.HAPBatch(Ns, Ls, damping=0.6, device=DEV)
    bt.set_preferences([x[2] for x in insts])
    for b, (_, S32, _) in enumerate(insts):
        bt.set_similarity(b, torch.from_numpy(S32).to(DEV))
    ms = bt.tune()
    assert ms > 0 and bt.query(8) in (2, 4, 6, 8, 12, 16) and bt.tile["elems_per_thread"] in (8, 16)
    bt.iterate(4)
    for b, (_, S32, prefs) in enumerate(insts):
        ref = H.run(H.level_similarities(S32.astype(np.float64), prefs.astype(np.float64)), 4, 0.6, H.PAPER)
        errs = _errs(bt.get_state(b), ref)
        assert all(e <= TOL for e in errs.values()), (b, errs)
    bt.close()


def test_batch_build_similarity_tensor_cores():
    from paper_1403_7394_gb300 import hap
    Ns, Ls = [250, 1030, 64], [2, 3, 2]
    insts = _instances(Ns, Ls, seed=3, d=32)
    X = torch.from_numpy(np.concatenate([x[0] for x in insts])).to(DEV)
    bt = hap.HAPBatch(Ns, Ls, damping=0.5, device=DEV)
    bt.set_preferences([x[2] for x in insts])
    bt.build_similarity(X, mode="bf16_split")
    bt.iterate(3)
    for b, (X32, _, prefs) in enumerate(insts):
        ctx = hap.HAP(Ns[b], Ls[b], prefs=prefs, damping=0.5, device=DEV)
        ctx.build_similarity(torch.from_numpy(X32).to(DEV), mode="bf16_split")
        ctx.iterate(3)
        errs = _errs(bt.get_state(b), ctx.get_state())
        assert all(e <= TOL for e in errs.values()), (b, errs)
        ctx.close()
    bt.close()


@pytest.mark.parametrize("Ns,Ls,tile", [([2600, 3100, 1500, 40], [3, 2, 4, 2], 0),     # 6, 7, 3, 1 warps per row
                                        ([2600, 3100, 1500, 40], [3, 2, 4, 2], 8),     # 11, 13, 6, 1 at 8 columns
                                        ([700, 2000, 150], [9, 2, 10], 0)])          # > 8 levels: 8 columns per thread
def test_batch_row_group_shapes(Ns, Ls, tile, report):
    """Row groups of every width (1..13 warps), at 16 and 8 columns per
    thread (8 by hand, or because an instance has more than 8 levels),
    against single-instance runs."""
    from paper_1403_7394_gb300 import hap
    insts = _instances(Ns, Ls, seed=40)
    bt = hap.HAPBatch(Ns, Ls, damping=0.5, device=DEV)
    bt.set_preferences([x[2] for x in insts])
    for b, (_, S32, _) in enumerate(insts):
        bt.set_similarity(b, torch.from_numpy(S32).to(DEV))
    if tile:
        bt.set_tile(tile)
    assert bt.tile["elems_per_thread"] == (tile or (16 if max(Ls) <= 8 else 8))
    bt.iterate(5)
    worst = 0.0
    for b, (_, S32, prefs) in enumerate(insts):
        ctx = hap.HAP(Ns[b], Ls[b], prefs=prefs, damping=0.5, device=DEV)
        ctx.set_similarity(torch.from_numpy(S32).to(DEV))
        ctx.iterate(5)
        errs = _errs(bt.get_state(b), ctx.get_state())
        worst = max(worst, max(errs.values()))
        assert all(e <= TOL for e in errs.values()), (b, errs)
        ctx.close()
    report(worst=worst, tile=bt.tile)
    bt.close()


def test_batch_tile_width_refused_beyond_8_levels():
    from paper_1403_7394_gb300 import hap
    bt = hap.HAPBatch([100, 200], [9, 2], damping=0.5, device=DEV)
    with pytest.raises(hap.HapError) as e:
        bt.set_tile(16)
    assert e.value.code == hap.HAP_EUNSUPPORTED
    with pytest.raises(hap.HapError) as e:
        bt.set_tile(12)
    assert e.value.code == hap.HAP_EINVAL
    bt.close()


def test_batch_many_items_per_cta(report):
    """More items than CTAs, so every CTA walks several (instance, band) items
    whose row groups differ in width (1..2 warps here) and level count; after
    the tuner, sampled instances against single-instance runs."""
    from paper_1403_7394_gb300 import hap
    rng = np.random.default_rng(11)
    B = 400
    Ns = [int(x) for x in rng.integers(30, 900, size=B)]
    Ls = [int(x) for x in rng.integers(1, 5, size=B)]
    insts = _instances(Ns, Ls, seed=500)
    bt = hap.HAPBatch(Ns, Ls, damping=0.5, device=DEV)
    bt.set_preferences([x[2] for x in insts])
    for b, (_, S32, _) in enumerate(insts):
        bt.set_similarity(b, torch.from_numpy(S32).to(DEV))
    bt.tune()
    bt.iterate(4)
    worst = 0.0
    for b in rng.choice(B, 12, replace=False):
        _, S32, prefs = insts[b]
        ctx = hap.HAP(Ns[b], Ls[b], prefs=prefs, damping=0.5, device=DEV)
        ctx.set_similarity(torch.from_numpy(S32).to(DEV))
        ctx.iterate(4)
        errs = _errs(bt.get_state(int(b)), ctx.get_state())
        worst = max(worst, max(errs.values()))
        assert all(e <= TOL for e in errs.values()), (b, errs)
        ctx.close()
    report(worst=worst, items_per_cta=bt.query(8))
    bt.close()


def test_batch_bf16_storage():
    """Batched instances with BF16-stored S equal single-instance runs with
    BF16-stored S (the same rounding of s, the same arithmetic)."""
    from paper_1403_7394_gb300 import hap
    Ns, Ls = [700, 2300, 150], [3, 2, 4]
    insts = _instances(Ns, Ls, seed=71)
    bt = hap.HAPBatch(Ns, Ls, damping=0.5, device=DEV, s_dtype="bf16")
    bt.set_preferences([x[2] for x in insts])
    for b, (_, S32, _) in enumerate(insts):
        bt.set_similarity(b, torch.from_numpy(S32).to(DEV))
    bt.iterate(5)
    for b, (_, S32, prefs) in enumerate(insts):
        ctx = hap.HAP(Ns[b], Ls[b], prefs=prefs, damping=0.5, device=DEV, s_dtype="bf16")
        ctx.set_similarity(torch.from_numpy(S32).to(DEV))
        ctx.iterate(5)
        errs = _errs(bt.get_state(b), ctx.get_state())
        assert all(e <= TOL for e in errs.values()), (b, errs)
        ctx.close()
    bt.close()
