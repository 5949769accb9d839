"""The allocation-free entry point (hap_iterate_noalloc), for callers that
cannot allocate device memory themselves, against the context-based entry
point on the same problem: two calls in a row (the second resumes where the
first stopped) must agree with hap_iterate within the message tolerance of
the parity tests.  Collected last on purpose."""
import numpy as np
import pytest
import torch

from oracle import hap_oracle as H
from paper_1403_7394_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = 1e-4


def _padded(x, shape, fill=0.0):
    out = torch.full(shape, fill, dtype=torch.float32, device=DEV)
    out[..., : x.shape[-1]] = torch.as_tensor(x, dtype=torch.float32, device=DEV)
    return out


@pytest.mark.parametrize("c_mode", ["paper", "fixed"])
def test_noalloc_matches_context_on_two_calls(c_mode):
    from paper_1403_7394_gb300 import hap
    N, L, lam = 1000, 3, 0.5
    X, _ = W.gmm_points(N, 2, 6, sigma=0.6, seed=77, means="uniform", mean_scale=10.0)
    S32 = H.neg_sq_euclidean(X).astype(np.float32)
    p = np.float32(H.median_preference(S32.astype(np.float64)))
    prefs = np.array([p, 1.5 * p, 2.0 * p], dtype=np.float32)
    ld = (N + 31) // 32 * 32

    ctx = hap.HAP(N, L, prefs=prefs, damping=lam, device=DEV, c_mode=c_mode)
    ctx.set_similarity(torch.from_numpy(S32).to(DEV))

    S = _padded(S32, (N, ld))
    pref = _padded(np.repeat(prefs[:, None], N, axis=1), (L, ld))
    A = torch.zeros((L, N, ld), dtype=torch.float32, device=DEV)
    R = torch.zeros_like(A)
    c = torch.zeros((L, ld), dtype=torch.float32, device=DEV)
    tau = torch.zeros_like(c)
    phi = torch.zeros_like(c)

    t = 0
    for n in (5, 7):  # two calls in a row; the second resumes at t = 5
        hap.iterate_noalloc(N, L, lam, c_mode, S, pref, A, R, c, tau, phi, t0=t, n=n)
        t += n
        ctx.iterate(n)
        ref = ctx.get_state()
        got = {"A": A[:, :, :N], "R": R[:, :, :N], "c": c[:, :N], "tau": tau[:, :N], "phi": phi[:, :N]}
        for k, v in got.items():
            err = H.message_rel_error(v.cpu().numpy().astype(np.float64), ref[k].cpu().numpy().astype(np.float64))
            assert err <= TOL, (t, k, err)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1403_7394_gb300 import hap
    N, L = 8192, 4  # L * ld = 32768 > 16384
    ld = N
    S = torch.zeros((N, ld), dtype=torch.float32, device=DEV)
    pref = torch.zeros((L, ld), dtype=torch.float32, device=DEV)
    A = torch.zeros((L, N, ld), dtype=torch.float32, device=DEV)
    R = torch.zeros_like(A)
    v = [torch.zeros((L, ld), dtype=torch.float32, device=DEV) for _ in range(3)]
    with pytest.raises(hap.HapError) as ei:
        hap.iterate_noalloc(N, L, 0.5, "paper", S, pref, A, R, *v, t0=0, n=1)
    assert ei.value.code == hap.HAP_EUNSUPPORTED
    assert hap.lib.hap_noalloc_scratch_bytes() > 0
