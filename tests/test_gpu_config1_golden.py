"""Free-running parity at full size: the 8192-point, 64-D, 64-component
mixture with L = 4 levels, lambda = 0.5 and 300 iterations, run by the CUDA
path (through the C ABI, in the launch shape the benchmark uses) from
Algorithm 1's start and compared with the FP64 reference's own run of the
same problem.

The reference results are stored in tests/golden/config1_free_running_*.npz
by tests/golden/make_config1_free_running.py (FP64 reference only).  Both
sides consume the same float32 similarity: it is rebuilt here on the host
with the reference's fixed-order formula and its SHA-256 must equal the one
the reference run stored.

Checked at every stored checkpoint t: the exemplars of Eq. 2.8 and the
message error err(X) = max|X_gpu - X_ref| / max(max|X_ref|, 1) on 4096
sampled alpha and rho entries and on c, tau, phi of 512 sampled points,
reported per checkpoint with the first t at which it exceeds 1e-4.

Required in both c modes: through t = 30 (the paper's iteration count, §4.1)
every message within 1e-4, and identical exemplars at every level at t = 30.
Before that the assignment is still changing for thousands of points and an
argmax can be a near-tie that FP32 and FP64 decide differently (measured: one
point of 8192 at level 2 at t = 2 in the "paper" mode while the messages
agree to 7e-8), so up to 0.1 % of the points per level may differ there.  With
Eq. 2.6 as printed ("paper") the run is contractive: also every checkpoint
to t = 300 within 1e-4 and identical exemplars and net similarity at t = 300
(measured on GB300: at most 5.4e-6; every point ends as its own exemplar at
every level, the degenerate outcome of the undamped c feedback).  With c
fixed the FP64 run itself has not converged by t = 300 (argmax margins down
to 1e-3, thousands of exemplars changing between checkpoints), so rounding
differences grow until the two runs decorrelate: measured 1.3e-5 at t = 30,
above 1e-4 first at the t = 50 checkpoint (1e-2, 3 exemplars differ), O(1)
from t = 75.  That is the conditioning of the iteration (one iteration from
the same state stays near 1e-7 in the teacher-forced tests), so beyond t = 30
it is reported, not gated.
"""
import importlib.util
import os

import numpy as np
import pytest
import torch


pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")
DEV = "cuda:0"


def _maker():
    spec = importlib.util.spec_from_file_location("make_config1", os.path.join(GOLDEN, "make_config1_free_running.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.fixture(scope="module")
def similarity():
    """(S float32 on the device, preference, SHA-256 of S) rebuilt from the
    seeded points."""
    mk = _maker()
    X, S32, pref, digest = mk.inputs()
    S = torch.from_numpy(S32).to(DEV)
    del S32
    return S, pref, digest


def _err(got, want, scale):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    fin = np.isfinite(want)
    if not np.array_equal(np.isfinite(got), fin) or not np.array_equal(got[~fin], want[~fin]):
        return float("inf")
    if not fin.any():
        return 0.0
    return float(np.max(np.abs(got[fin] - want[fin])) / max(scale, 1.0))


@pytest.mark.parametrize("c_mode", ["paper", "fixed"])
def test_config1_free_running_300_iterations(similarity, c_mode, report):
    from paper_1403_7394_gb300 import hap
    S, pref, digest = similarity
    z = np.load(os.path.join(GOLDEN, f"config1_free_running_{c_mode}.npz"))
    assert str(z["s_sha256"]) == digest, "the rebuilt similarity differs from the reference run's"
    assert np.float32(z["pref"]) == pref
    N, L, lam = int(z["N"]), int(z["L"]), float(z["lam"])
    lv, si, sj, pts = (torch.from_numpy(z[k].astype(np.int64)).to(DEV)
                       for k in ("sample_level", "sample_row", "sample_col", "sample_points"))
    ctx = hap.HAP(N, L, prefs=np.full(L, pref, dtype=np.float32), damping=lam, device=DEV, c_mode=c_mode)
    ctx.set_similarity(S)
    curve, t_done = [], 0
    for k, t in enumerate(z["checkpoints"].tolist()):
        ctx.iterate(t - t_done)
        t_done = t
        g = ctx.get_state()
        e = ctx.exemplars().cpu().numpy()
        row = {"t": t,
               "A": _err(g["A"][lv, si, sj].cpu().numpy(), z["A"][k], z["scale_A"][k]),
               "R": _err(g["R"][lv, si, sj].cpu().numpy(), z["R"][k], z["scale_R"][k])}
        for f in ("c", "tau", "phi"):
            want = z[f][k]
            fin = want[np.isfinite(want)]
            row[f] = _err(g[f][:, pts].cpu().numpy(), want, float(np.max(np.abs(fin))) if fin.size else 1.0)
        row["exemplar_mismatches"] = [int(np.sum(e[l] != z["e"][k][l])) for l in range(L)]
        row["exemplars"] = [int(np.unique(e[l]).size) for l in range(L)]
        curve.append(row)
        del g
    over = [r["t"] for r in curve if max(r[f] for f in ("A", "R", "c", "tau", "phi")) > 1e-4]
    final = curve[-1]
    e_ref = z["e"][-1].astype(np.int32)
    e_gpu = ctx.exemplars().cpu().numpy()
    ns_gpu, ns_ref = ctx.net_similarity(), z["net_similarity"]
    report(c_mode=c_mode, curve=curve, first_t_above_1e4=over[0] if over else None,
           exemplars_ref=[int(np.unique(x).size) for x in e_ref], ns_gpu=list(map(float, ns_gpu)),
           ns_ref=list(map(float, ns_ref)), min_margin_ref=[float(m) for m in z["margin_min"]])
    print({"c_mode": c_mode, "first_t_above_1e4": over[0] if over else None,
           "final_mismatches": final["exemplar_mismatches"]})
    ctx.close()
    for r in curve:
        if r["t"] <= 30:
            assert max(r[f] for f in ("A", "R", "c", "tau", "phi")) <= 1e-4, r
            assert max(r["exemplar_mismatches"]) <= N // 1000, r
        if r["t"] == 30:
            assert r["exemplar_mismatches"] == [0] * L, r
    if c_mode == "paper":
        assert not over, over
        np.testing.assert_array_equal(e_gpu, e_ref)
        assert final["exemplar_mismatches"] == [0] * L
        np.testing.assert_allclose(ns_gpu, ns_ref, rtol=1e-9)
