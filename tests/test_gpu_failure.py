"""Failure detection on the GPU without a GPU fault, and the debug checks.

* Bounded waits: a context whose wait limit is 1 ns cannot see its first TMA
  ring stage land in time, so the row pass gives up, lets its own copies land
  and returns; the next synchronising call reports HAP_ETIMEOUT.  The CUDA
  context stays usable: the same library context, given its default limit
  and a new state, then runs bit for bit like a fresh one.  Cluster size 1
  only: the expiry path there involves no peer CTA.
* The batched row pass (one persistent launch over many instances) the same
  way: with a 1 ns limit its waits give up, nothing more is issued, every CTA
  lets its own copies land and leaves; HAP_ETIMEOUT is reported and the batch,
  given its default limit and new similarities, runs bit for bit like a fresh
  one.
* debug_bounds: a non-finite similarity is refused (HAP_EINVAL), and the row
  pass's index checks change no bit of the result.
"""
import numpy as np
import pytest
import torch

from test_gpu_parity import DEV, hap_mod, make_ctx, problem

pytestmark = pytest.mark.gpu

HAP_EINVAL, HAP_ETIMEOUT = -1, -5


def _states_equal(a, b):
    ga, gb = a.get_state(), b.get_state()
    for k in ("A", "R", "c", "tau", "phi"):
        assert torch.equal(ga[k], gb[k]), k


@pytest.mark.parametrize("opt", [{"cluster_size": 1}, {"cluster_size": 1, "col_sums": "tmem"},
                                 {"cluster_size": 1, "col_sums": "smem", "elems_per_thread": 16}])
def test_wait_expiry_reports_timeout_and_the_context_recovers(opt):
    hap = hap_mod()
    N, L, lam = 2048, 3, 0.5
    S32, prefs, _ = problem(N, L, seed=3)
    ctx = make_ctx(N, L, prefs, lam, S32, wait_limit_ns=1, **opt)
    assert ctx.query(2) == 1  # HAP_Q_CLUSTER_SIZE
    ctx.iterate(3)
    with pytest.raises(hap.HapError) as err:
        ctx.sync()
    assert err.value.code == HAP_ETIMEOUT
    torch.cuda.synchronize()  # no sticky CUDA error: the kernels returned
    # the error stays reported until the context gets a new state
    with pytest.raises(hap.HapError):
        ctx.sync()
    ctx.set_wait_limit(0)
    ctx.set_similarity(torch.from_numpy(S32).to(DEV))
    ctx.iterate(4)
    ctx.sync()
    fresh = make_ctx(N, L, prefs, lam, S32, **opt)
    fresh.iterate(4)
    _states_equal(ctx, fresh)
    ctx.close()
    fresh.close()


def test_batched_wait_expiry_reports_timeout_and_the_batch_recovers():
    hap = hap_mod()
    Ns, Ls = [1500, 700, 3000, 90], [3, 2, 2, 4]
    probs = [problem(n, l, seed=20 + q) for q, (n, l) in enumerate(zip(Ns, Ls))]

    def make():
        bt = hap.HAPBatch(Ns, Ls, damping=0.5, device=DEV)
        bt.set_preferences([p[1] for p in probs])
        for b, p in enumerate(probs):
            bt.set_similarity(b, torch.from_numpy(p[0]).to(DEV))
        return bt

    bt = make()
    bt.set_wait_limit(1)
    bt.iterate(3)  # a direct launch, then graph replays carrying the 1 ns limit
    with pytest.raises(hap.HapError) as err:
        bt.sync()
    assert err.value.code == HAP_ETIMEOUT
    torch.cuda.synchronize()  # no sticky CUDA error: every CTA returned
    bt.set_wait_limit(0)
    for b, p in enumerate(probs):  # a new state clears the report
        bt.set_similarity(b, torch.from_numpy(p[0]).to(DEV))
    bt.iterate(4)
    bt.sync()
    fresh = make()
    fresh.iterate(4)
    fresh.sync()
    for b in range(len(Ns)):
        ga, gb = bt.get_state(b), fresh.get_state(b)
        for k in ("A", "R", "c", "tau", "phi"):
            assert torch.equal(ga[k], gb[k]), (b, k)
    bt.close()
    fresh.close()


@pytest.mark.parametrize("s_dtype", ["f32", "bf16"])
@pytest.mark.parametrize("bad", [float("nan"), float("-inf"), float("inf")])
def test_debug_bounds_refuses_non_finite_similarity(bad, s_dtype):
    hap = hap_mod()
    N, L = 300, 2
    S32, prefs, _ = problem(N, L, seed=4)
    S_bad = S32.copy()
    S_bad[17, 250] = bad
    ctx = hap.HAP(N, L, prefs=prefs, damping=0.5, device=DEV, s_dtype=s_dtype, debug_bounds=True)
    with pytest.raises(hap.HapError) as err:
        ctx.set_similarity(torch.from_numpy(S_bad).to(DEV))
    assert err.value.code == HAP_EINVAL
    # the diagonal is not a similarity (the preferences replace it)
    S_diag = S32.copy()
    S_diag[5, 5] = bad
    ctx.set_similarity(torch.from_numpy(S_diag).to(DEV))
    ctx.iterate(2)
    ctx.sync()
    # points with a NaN coordinate give a NaN similarity row
    X = torch.randn(N, 8, device=DEV)
    X[9, 3] = float("nan")
    with pytest.raises(hap.HapError) as err:
        ctx.build_similarity(X, mode="f32")
    assert err.value.code == HAP_EINVAL
    X[9, 3] = 0.0
    ctx.build_similarity(X, mode="bf16_split")
    ctx.close()
    # without the option the library takes the caller's word for it
    plain = hap.HAP(N, L, prefs=prefs, damping=0.5, device=DEV, s_dtype=s_dtype)
    plain.set_similarity(torch.from_numpy(S_bad).to(DEV))
    plain.close()


@pytest.mark.parametrize("opt", [{}, {"cluster_size": 2, "col_sums": "tmem"}, {"elems_per_thread": 8}])
def test_debug_bounds_changes_no_bits(opt):
    N, L, lam = 1500, 3, 0.5
    S32, prefs, _ = problem(N, L, seed=6)
    a = make_ctx(N, L, prefs, lam, S32, debug_bounds=True, **opt)
    b = make_ctx(N, L, prefs, lam, S32, **opt)
    a.iterate(6)
    b.iterate(6)
    a.sync()
    _states_equal(a, b)
    np.testing.assert_array_equal(a.exemplars().cpu().numpy(), b.exemplars().cpu().numpy())
