"""The allocation-free entry point (hap_iterate_noalloc), for callers that
cannot allocate device memory themselves, against the context-based entry
point on the same problem: two calls in a row (the second resumes where the
first stopped) must agree with hap_iterate within the message tolerance of
the parity tests.  Also checked: FP32 and BF16 similarity, the largest size
its fixed scratch takes (L * ld = 16384), one iteration per call against the
FP64 reference directly, and that a call leaves the device's free memory
unchanged.  Collected last on purpose."""
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


def _problem(N, L, seed=77):
    X, _ = W.gmm_points(N, 2, 6, sigma=0.6, seed=seed, means="uniform", mean_scale=10.0)
    S32 = H.neg_sq_euclidean(X).astype(np.float32)
    p = np.float32(H.median_preference(S32[:512, :512].astype(np.float64)))
    prefs = np.array([p * (1.0 + 0.5 * l) for l in range(L)], dtype=np.float32)
    return S32, prefs


def _buffers(N, L, S32, prefs, s_dtype):
    ld = (N + 31) // 32 * 32
    S = _padded(S32, (N, ld))
    if s_dtype == "bf16":
        S = S.to(torch.bfloat16)
    pref = _padded(np.repeat(prefs[:, None], N, axis=1), (L, ld))
    A = torch.zeros((L, N, ld), dtype=torch.float32, device=DEV)
    R = torch.zeros_like(A)
    c = torch.zeros((L, ld), dtype=torch.float32, device=DEV)
    return S, pref, A, R, c, torch.zeros_like(c), torch.zeros_like(c)


@pytest.mark.parametrize("N,L,s_dtype", [(1000, 3, "f32"), (1000, 3, "bf16"), (4096, 4, "f32")])
@pytest.mark.parametrize("c_mode", ["paper", "fixed"])
def test_noalloc_matches_context_on_two_calls(N, L, s_dtype, c_mode):
    from paper_1403_7394_gb300 import hap
    lam = 0.5
    S32, prefs = _problem(N, L)
    ctx = hap.HAP(N, L, prefs=prefs, damping=lam, device=DEV, c_mode=c_mode, s_dtype=s_dtype)
    ctx.set_similarity(torch.from_numpy(S32).to(DEV))
    S, pref, A, R, c, tau, phi = _buffers(N, L, S32, prefs, s_dtype)
    t = 0
    for n in (5, 7):  # two calls in a row; the second resumes at t = 5
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        hap.iterate_noalloc(N, L, lam, c_mode, S, pref, A, R, c, tau, phi, t0=t, n=n)
        torch.cuda.synchronize()
        if t > 0:  # after the first call on the device, the device's free memory is unchanged
            assert torch.cuda.mem_get_info()[0] == free0
        t += n
        ctx.iterate(n)
        ref = ctx.get_state()
        got = {"A": A[:, :, :N], "R": R[:, :, :N], "c": c[:, :N], "tau": tau[:, :N], "phi": phi[:, :N]}
        for k, v in got.items():
            err = H.message_rel_error(v.cpu().numpy().astype(np.float64), ref[k].cpu().numpy().astype(np.float64))
            assert err <= TOL, (t, k, err)
    ctx.close()


@pytest.mark.parametrize("c_mode", ["paper", "fixed"])
def test_noalloc_one_iteration_per_call_against_the_reference(c_mode):
    """From a reference state rounded to FP32, each call of one iteration
    must give the reference's next state (Eqs. 2.1-2.6 with damping)."""
    from paper_1403_7394_gb300 import hap
    N, L, lam = 700, 3, 0.5
    S32, prefs = _problem(N, L, seed=5)
    S_ref = H.level_similarities(S32.astype(np.float64), prefs.astype(np.float64))
    st = H.run(S_ref, 3, lam, c_mode)
    S, pref, A, R, c, tau, phi = _buffers(N, L, S32, prefs, "f32")
    A[:, :, :N] = torch.from_numpy(st.A.astype(np.float32)).to(DEV)
    R[:, :, :N] = torch.from_numpy(st.R.astype(np.float32)).to(DEV)
    c[:, :N] = torch.from_numpy(st.c.astype(np.float32)).to(DEV)
    cur = H.HAPState(st.A.astype(np.float32).astype(np.float64), st.R.astype(np.float32).astype(np.float64),
                     st.c.astype(np.float32).astype(np.float64), st.tau, st.phi, st.t)
    for _ in range(2):
        hap.iterate_noalloc(N, L, lam, c_mode, S, pref, A, R, c, tau, phi, t0=cur.t, n=1)
        cur = H.step(S_ref, cur, lam, c_mode)
        got = {"A": A[:, :, :N], "R": R[:, :, :N], "c": c[:, :N], "tau": tau[:, :N], "phi": phi[:, :N]}
        for k, v in got.items():
            err = H.message_rel_error(v.cpu().numpy().astype(np.float64), getattr(cur, k))
            assert err <= TOL, (cur.t, k, err)


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
    n, l = 64, 2  # messages must be float32 tensors on the similarity's device
    small = _buffers(n, l, np.zeros((n, n), np.float32), np.zeros(l, np.float32), "f32")
    with pytest.raises(ValueError):
        hap.iterate_noalloc(n, l, 0.5, "paper", small[0], small[1], small[2].double(), *small[3:], t0=0, n=1)
