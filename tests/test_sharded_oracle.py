"""Row-sharded HAP with one sum all-reduce per iteration (the multi-GPU
design: each shard owns a set of rows, only column statistics and owned
vectors cross shards), run as two gloo ranks on CPU and compared with the
unsharded reference."""
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


def _problem():
    X, _ = W.gmm_points(N, 2, 4, sigma=0.6, seed=13)
    S0 = H.neg_sq_euclidean(X)
    p = H.median_preference(S0)
    return H.level_similarities(S0, [p, 1.5 * p, 2.0 * p])


def _rank_main(rank, world, init_file, c_mode, restart_at, out_dir):
    dist.init_process_group("gloo", init_method=f"file://{init_file}", rank=rank, world_size=world)

    def allreduce(x):
        t = torch.from_numpy(np.ascontiguousarray(x))
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return t.numpy()

    S = _problem()
    rows = np.arange(rank, N, world)  # interleaved ownership, as the GPU's clusters own rows
    st = H.init_state(L, N)
    carry = None
    for t in range(T):
        if t == restart_at:
            carry = None  # a restarted shard rebuilds the column statistics
        st, carry = H.step_sharded(S, st, rows, LAM, c_mode, allreduce, carry)
    np.savez(os.path.join(out_dir, f"r{rank}.npz"), A=st.A[:, rows], R=st.R[:, rows], c=st.c, tau=st.tau[:, rows],
             phi=st.phi, rows=rows)
    dist.destroy_process_group()


@pytest.mark.parametrize("c_mode,restart_at", [("paper", -1), ("fixed", -1), ("paper", 5)])
def test_two_rank_sharded_step_matches_unsharded(c_mode, restart_at):
    world = 2
    with tempfile.TemporaryDirectory() as d:
        init_file = os.path.join(d, "init")
        mp.start_processes(_rank_main, args=(world, init_file, c_mode, restart_at, d), nprocs=world,
                           join=True, start_method="spawn")
        ref = H.run(_problem(), T, LAM, c_mode)
        A = np.zeros_like(ref.A)
        R = np.zeros_like(ref.R)
        tau = np.zeros_like(ref.tau)
        for r in range(world):
            z = np.load(os.path.join(d, f"r{r}.npz"))
            A[:, z["rows"]] = z["A"]
            R[:, z["rows"]] = z["R"]
            tau[:, z["rows"]] = z["tau"]
            np.testing.assert_allclose(z["c"], ref.c, rtol=0, atol=1e-9)
            np.testing.assert_allclose(z["phi"], ref.phi, rtol=0, atol=1e-9)
        scale = max(1.0, np.abs(ref.R).max())
        assert np.abs(A - ref.A).max() <= 1e-12 * scale
        assert np.abs(R - ref.R).max() <= 1e-12 * scale
        assert H.message_rel_error(tau, ref.tau) <= 1e-12
