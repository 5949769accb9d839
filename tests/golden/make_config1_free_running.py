#!/usr/bin/env python
"""Writes the expected results of the 8192-point, 64-D mixture workload run
free for 300 iterations by the FP64 reference (HAP, §2 Eqs. 2.1-2.6 and 2.8,
Algorithm 1, Jacobi level schedule).

Only the FP64 reference (``oracle/``) and the seeded point generators are
used; nothing here comes from the CUDA library.

Inputs, rebuilt bit for bit by the GPU test on any IEEE-754 machine:
  * X: 8192 points in 64-D, 64 components, means ~ N(0, 4 I), sigma = 1,
    seed 0, rounded to float32 (the points the library receives);
  * S: the fixed-order float64 similarity of those points, rounded to
    float32; its SHA-256 is stored so that a test can prove it fed the
    same bits;
  * one preference at every one of the L = 4 levels: the median of the
    N(N-1) off-diagonal float32 similarities computed in float64, rounded
    to float32;
  * lambda = 0.5, 300 iterations, c mode "paper" (Eq. 2.6 as printed) or
    "fixed" (c = 0).

Stored per checkpoint t: the exemplars of Eq. 2.8 (int16), 4096 sampled
message entries of alpha and rho (512 of them on the diagonal), the largest
|alpha| and |rho| over the whole tensors (the scale of the message error),
and c, tau, phi of 512 sampled points; at t = 300 also the net similarity and,
per level, the smallest and the 1 % quantile of the rows' argmax margins
(best minus second best alpha + rho), which show how far rounding would have
to move a message to change an exemplar.

    python tests/golden/make_config1_free_running.py [paper|fixed ...]
    python tests/golden/make_config1_free_running.py --trim FILE.npz ...

Takes about an hour and 16 GB per mode on one host core.  --trim rewrites a
file written by an earlier version of this script (which also kept the full
final c, tau, phi and every row's margin) in the current format.
"""
from __future__ import annotations

import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import hap_oracle as H  # noqa: E402
from paper_1403_7394_gb300 import workloads as W  # noqa: E402

N, D, L, LAM, T = 8192, 64, 4, 0.5, 300
CHECKPOINTS = (1, 2, 3, 5, 10, 20, 30, 50, 75, 100, 150, 200, 250, 300)
N_SAMPLES, N_DIAG, N_POINTS = 4096, 512, 512


def inputs():
    """(X float32, S float32, preference float32, SHA-256 of S's bytes)."""
    X, _ = W.config1(seed=0)
    X = X.astype(np.float32)
    S = H.neg_sq_euclidean_fixed_order(X.astype(np.float64)).astype(np.float32)
    pref = np.float32(H.median_preference(S.astype(np.float64)))
    return X, S, pref, hashlib.sha256(S.tobytes()).hexdigest()


def sample_indices():
    """Seeded (level, row, column) message samples and sampled points."""
    rng = np.random.default_rng(12345)
    n_off = N_SAMPLES - N_DIAG
    lv = rng.integers(0, L, N_SAMPLES)
    i = rng.integers(0, N, N_SAMPLES)
    j = rng.integers(0, N, N_SAMPLES)
    j[n_off:] = i[n_off:]
    pts = np.sort(rng.choice(N, N_POINTS, replace=False))
    return lv.astype(np.int32), i.astype(np.int32), j.astype(np.int32), pts.astype(np.int32)


def margin_summary(margin):
    """Per level: the smallest and the 1 % quantile of the argmax margins."""
    return {"margin_min": margin.min(axis=1), "margin_q01": np.quantile(margin, 0.01, axis=1)}


def trim(path):
    """Rewrites a file of an earlier version of this script in the current
    format: the same stored values, without the full final c, tau, phi and
    with the margins summarised."""
    z = dict(np.load(path))
    for k in ("c_final", "tau_final", "phi_final"):
        z.pop(k, None)
    if "margin" in z:
        z.update(margin_summary(z.pop("margin")))
    np.savez_compressed(path, **z)


def main(modes):
    t_all = time.time()
    X, S32, pref, digest = inputs()
    print(f"inputs ready ({time.time() - t_all:.0f} s): pref {pref!r}, S sha256 {digest}", flush=True)
    S_ref = H.level_similarities(S32.astype(np.float64), np.full(L, pref, dtype=np.float64))
    del S32
    lv, si, sj, pts = sample_indices()
    for mode in modes:
        rec = {k: [] for k in ("t", "e", "A", "R", "scale_A", "scale_R", "c", "tau", "phi")}
        t0 = time.time()

        def cb(st):
            if st.t not in CHECKPOINTS:
                return
            rec["t"].append(st.t)
            rec["e"].append(H.exemplars(st.A, st.R).astype(np.int16))
            rec["A"].append(st.A[lv, si, sj])
            rec["R"].append(st.R[lv, si, sj])
            rec["scale_A"].append(float(np.max(np.abs(st.A))))
            rec["scale_R"].append(float(np.max(np.abs(st.R))))
            rec["c"].append(st.c[:, pts])
            rec["tau"].append(st.tau[:, pts])
            rec["phi"].append(st.phi[:, pts])
            print(f"{mode} t={st.t} ({time.time() - t0:.0f} s) exemplars per level "
                  f"{[len(np.unique(x)) for x in rec['e'][-1]]}", flush=True)

        st = H.run(S_ref, T, LAM, mode, callback=cb)
        e = H.exemplars(st.A, st.R)
        ns = H.net_similarity(S_ref, e)
        V = st.A + st.R
        top2 = np.partition(V, N - 2, axis=2)[:, :, N - 2:]
        margin = (top2[:, :, 1] - top2[:, :, 0]).astype(np.float32)
        del V, top2
        out = os.path.join(HERE, f"config1_free_running_{mode}.npz")
        np.savez_compressed(
            out, N=N, d=D, L=L, lam=LAM, T=T, c_mode=mode, pref=pref, s_sha256=digest,
            checkpoints=np.array(rec["t"], dtype=np.int32), e=np.stack(rec["e"]),
            sample_level=lv, sample_row=si, sample_col=sj, sample_points=pts,
            A=np.stack(rec["A"]), R=np.stack(rec["R"]),
            scale_A=np.array(rec["scale_A"]), scale_R=np.array(rec["scale_R"]),
            c=np.stack(rec["c"]), tau=np.stack(rec["tau"]), phi=np.stack(rec["phi"]),
            net_similarity=ns, **margin_summary(margin), oracle_seconds=time.time() - t0)
        print(f"{mode}: wrote {out} ({os.path.getsize(out)} bytes, {time.time() - t0:.0f} s); "
              f"NS {ns.tolist()}", flush=True)


if __name__ == "__main__":
    if sys.argv[1:2] == ["--trim"]:
        for f in sys.argv[2:]:
            trim(f)
    else:
        main(sys.argv[1:] or ["paper", "fixed"])
