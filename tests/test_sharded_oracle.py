"""Row-sharded HAP with one sum all-reduce per iteration (the multi-GPU
design: each shard owns a band of rows of S, alpha and rho, and only column
statistics and owned vectors cross shards), run as gloo ranks on CPU and
compared bit for bit with the unsharded reference summing its column sums in
the same shard order."""
import os
import tempfile

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import hap_oracle as H
from paper_1403_7394_gb300 import workloads as W

N, L, LAM, T = 60, 3, 0.5, 12
PREF_SCALE = (1.0, 1.5, 2.0)


def _points():
    X, _ = W.gmm_points(N, 2, 4, sigma=0.6, seed=13)
    return X


def _problem():
    S0 = H.neg_sq_euclidean(_points())
    p = H.median_preference(S0)
    return H.level_similarities(S0, [p * k for k in PREF_SCALE])


def _partition(world, layout):
    if layout == "interleaved":  # the GPU's clusters own rows g, g + G, ...
        return [np.arange(r, N, world) for r in range(world)]
    bounds = np.linspace(0, N, world + 1).astype(int)  # contiguous bands
    return [np.arange(bounds[r], bounds[r + 1]) for r in range(world)]


def _rank_main(rank, world, init_file, c_mode, restart_at, layout, out_dir):
    dist.init_process_group("gloo", init_method=f"file://{init_file}", rank=rank, world_size=world)

    def allreduce(x):
        t = torch.from_numpy(np.ascontiguousarray(x))
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return t.numpy()

    rows = _partition(world, layout)[rank]
    S0 = H.neg_sq_euclidean(_points())
    p = H.median_preference(S0)
    S_rows = H.level_similarity_rows(S0[rows], rows, [p * k for k in PREF_SCALE])
    del S0
    st = H.init_shard_state(L, N, rows)
    carry = None
    for t in range(T):
        if t == restart_at:
            carry = None  # a restarted shard rebuilds the column statistics
        st, carry = H.step_sharded(S_rows, st, rows, LAM, c_mode, allreduce, carry)
    np.savez(os.path.join(out_dir, f"r{rank}.npz"), A=st.A, R=st.R, c=st.c, tau=st.tau[:, rows],
             phi=st.phi, rows=rows)
    dist.destroy_process_group()


@pytest.mark.parametrize("c_mode,restart_at,layout", [("paper", -1, "interleaved"), ("fixed", -1, "interleaved"),
                                                      ("paper", 5, "interleaved"), ("fixed", -1, "bands")])
def test_two_rank_sharded_step_equals_unsharded(c_mode, restart_at, layout):
    world = 2
    with tempfile.TemporaryDirectory() as d:
        init_file = os.path.join(d, "init")
        mp.start_processes(_rank_main, args=(world, init_file, c_mode, restart_at, layout, d), nprocs=world,
                           join=True, start_method="spawn")
        ref = H.run(_problem(), T, LAM, c_mode, partition=_partition(world, layout))
        A = np.full_like(ref.A, np.nan)
        R = np.full_like(ref.R, np.nan)
        tau = np.full_like(ref.tau, np.nan)
        for r in range(world):
            z = np.load(os.path.join(d, f"r{r}.npz"))
            A[:, z["rows"]] = z["A"]
            R[:, z["rows"]] = z["R"]
            tau[:, z["rows"]] = z["tau"]
            np.testing.assert_array_equal(z["c"], ref.c)
            np.testing.assert_array_equal(z["phi"], ref.phi)
        np.testing.assert_array_equal(A, ref.A)
        np.testing.assert_array_equal(R, ref.R)
        np.testing.assert_array_equal(tau, ref.tau)


def test_partition_changes_only_the_summation_order():
    """The shard-ordered column sums are the same mathematical sum: the
    unsharded runs with and without a partition agree to rounding."""
    S = _problem()
    a = H.run(S, T, LAM, H.PAPER)
    b = H.run(S, T, LAM, H.PAPER, partition=_partition(3, "interleaved"))
    for f in ("A", "R", "c", "tau", "phi"):
        assert H.message_rel_error(getattr(b, f), getattr(a, f)) <= 1e-12
