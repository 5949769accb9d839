"""The stored results of the FP64 reference's free-running config-1 runs
(tests/golden/config1_free_running_*.npz) against facts that do not depend
on the reference's code: the similarity and preference they were computed on
(rebuilt here from the seeded points) and the first iteration's
responsibilities, which have a closed form (Eq. 2.1 with alpha = 0 and tau =
+inf at t = 1: rho = (1 - lambda)(s_ij - max_{k != j} s_ik))."""
import hashlib
import os

import numpy as np
import pytest

from oracle import hap_oracle as H
from paper_1403_7394_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MODES = ("paper", "fixed")


def _load(mode):
    return np.load(os.path.join(GOLDEN, f"config1_free_running_{mode}.npz"))


@pytest.fixture(scope="module")
def points():
    X, _ = W.config1(seed=0)
    return X.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("mode", MODES)
def test_first_iteration_closed_form(points, mode):
    z = _load(mode)
    assert int(z["checkpoints"][0]) == 1
    lam, pref = float(z["lam"]), float(z["pref"])
    rows = np.unique(z["sample_row"])
    S = H.neg_sq_euclidean_fixed_order(points, rows=rows).astype(np.float32).astype(np.float64)
    S[np.arange(rows.size), rows] = pref
    pos = {int(r): q for q, r in enumerate(rows)}
    want = np.empty(z["sample_row"].size)
    for n, (i, j) in enumerate(zip(z["sample_row"], z["sample_col"])):
        s = S[pos[int(i)]]
        others = np.delete(s, j)
        want[n] = (1.0 - lam) * (s[j] - others.max())
    np.testing.assert_allclose(z["R"][0], want, rtol=1e-12, atol=1e-12)
    # alpha after one iteration: the damped Eq. 2.2 / 2.3 update of alpha = 0
    assert np.all(z["A"][0][z["sample_row"] != z["sample_col"]] <= 0.0)


def test_similarity_and_preference_of_the_stored_runs(points):
    S32 = H.neg_sq_euclidean_fixed_order(points).astype(np.float32)
    digest = hashlib.sha256(S32.tobytes()).hexdigest()
    pref = np.float32(H.median_preference(S32.astype(np.float64)))
    for mode in MODES:
        z = _load(mode)
        assert str(z["s_sha256"]) == digest
        assert np.float32(z["pref"]) == pref
        assert int(z["N"]) == 8192 and int(z["L"]) == 4 and int(z["T"]) == 300 and float(z["lam"]) == 0.5
