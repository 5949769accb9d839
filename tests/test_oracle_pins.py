"""Pins of the FP64 reference against facts fixed by the paper and by
mathematics, independent of the reference's own code:

* worked examples derived by hand from Eqs. 2.1-2.7 under both level
  schedules (tests/golden),
* L = 1 with c fixed at 0 is flat affinity propagation (Frey & Dueck), written
  here separately with literal loops and literal sums,
* exhaustive search of exemplar sets on tiny inputs (net similarity),
* exact invariants: power-of-two scaling, permutation equivariance,
  self-consistency of converged assignments,
* library cross-checks (scipy distances, scikit-learn where installed).
"""
import itertools
import json
import os

import numpy as np
import pytest

from oracle import hap_oracle as H
from paper_1403_7394_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_n3.json")


def _arr(x):
    return np.array([[float("inf") if v == "inf" else v for v in row] for row in x], dtype=np.float64) \
        if np.ndim(x) == 2 else np.array(x, dtype=np.float64)


# ---------------------------------------------------------------- hand example
def _golden_cases():
    g = json.load(open(GOLDEN))
    for name, case in g["cases"].items():
        for t in (1, 2):
            if f"t{t}" in case:
                yield pytest.param(g, name, t, id=f"{name}-t{t}")


@pytest.mark.parametrize("g,name,t", list(_golden_cases()))
def test_hand_example(g, name, t):
    case = g["cases"][name]
    S = H.level_similarities(np.array(case.get("S_offdiag", g["S_offdiag"]), float), case["prefs"])
    st = H.init_state(S.shape[0], 3)
    for _ in range(t):
        st = H.step(S, st, g["lam"], case["c_mode"], case.get("schedule", H.JACOBI), case.get("kappa", 0.0))
    exp = case[f"t{t}"]
    for fld, val in exp.items():
        if fld == "e":
            np.testing.assert_array_equal(H.exemplars(st.A, st.R), np.array(val))
        elif fld == "ns":
            got = H.net_similarity(S, H.exemplars(st.A, st.R))
            np.testing.assert_array_equal(got, np.array(val, float))
        else:
            np.testing.assert_array_equal(getattr(st, fld), _arr(val), err_msg=f"{name} t{t} {fld}")


# ------------------------------------------------- flat AP special case (L = 1)
def textbook_ap(s, iterations, lam):
    """Frey & Dueck affinity propagation with literal loops and sums:
    r(i,k) = s(i,k) - max_{k' != k} [a(i,k') + s(i,k')]
    a(i,k) = min(0, r(k,k) + sum_{i' not in {i,k}} max(0, r(i',k)))   (i != k)
    a(k,k) = sum_{i' != k} max(0, r(i',k))
    both damped as lam*old + (1-lam)*new, r before a."""
    n = len(s)
    r = [[0.0] * n for _ in range(n)]
    a = [[0.0] * n for _ in range(n)]
    for _ in range(iterations):
        rn = [[0.0] * n for _ in range(n)]
        for i in range(n):
            for k in range(n):
                best = -float("inf")
                for kp in range(n):
                    if kp != k:
                        best = max(best, a[i][kp] + s[i][kp])
                rn[i][k] = s[i][k] - best
        r = [[lam * r[i][k] + (1 - lam) * rn[i][k] for k in range(n)] for i in range(n)]
        an = [[0.0] * n for _ in range(n)]
        for i in range(n):
            for k in range(n):
                if i != k:
                    tot = r[k][k]
                    for ip in range(n):
                        if ip != i and ip != k:
                            tot += max(0.0, r[ip][k])
                    an[i][k] = min(0.0, tot)
                else:
                    tot = 0.0
                    for ip in range(n):
                        if ip != k:
                            tot += max(0.0, r[ip][k])
                    an[i][k] = tot
        a = [[lam * a[i][k] + (1 - lam) * an[i][k] for k in range(n)] for i in range(n)]
    return np.array(a), np.array(r)


def _asymmetric(S0, seed):
    """A non-metric similarity (allowed by §2): S scaled row-wise by factors
    in [0.5, 1.5], so s_ij != s_ji."""
    f = np.random.default_rng(seed).uniform(0.5, 1.5, size=S0.shape[0])
    return S0 * f[:, None]


@pytest.mark.parametrize("seed,n,lam,T,asym", [(0, 12, 0.5, 25, False), (1, 17, 0.9, 40, False),
                                               (2, 9, 0.7, 60, True), (4, 14, 0.5, 30, True)])
def test_one_level_is_flat_affinity_propagation(seed, n, lam, T, asym):
    X, _ = W.gmm_points(n, 2, 3, sigma=0.7, seed=seed)
    S0 = H.neg_sq_euclidean(X)
    if asym:
        S0 = _asymmetric(S0, seed)
    p = H.median_preference(S0)
    S = H.level_similarities(S0, [p])
    st = H.run(S, T, lam, H.FIXED)
    a, r = textbook_ap(S[0].tolist(), T, lam)
    scale = max(np.abs(r).max(), 1.0)
    assert np.abs(st.R[0] - r).max() <= 1e-12 * scale
    assert np.abs(st.A[0] - a).max() <= 1e-12 * scale
    assert np.all(np.isinf(st.tau)) and np.all(st.phi == 0) and np.all(st.c == 0)


def test_flat_ap_matches_scikit_learn():
    sk = pytest.importorskip("sklearn.cluster")
    metrics = pytest.importorskip("sklearn.metrics")
    import warnings
    for seed in range(3):
        X, _ = W.gmm_points(60, 2, 4, sigma=0.5, seed=seed, means="uniform", mean_scale=10)
        S0 = H.neg_sq_euclidean(X)
        p = H.median_preference(S0)
        S = H.level_similarities(S0, [p])
        st = H.run(S, 400, 0.9, H.FIXED)
        e = H.exemplars(st.A, st.R)[0]
        Sk = S0.copy()
        np.fill_diagonal(Sk, p)
        with warnings.catch_warnings():
            warnings.simplefilter("ignore")
            ap = sk.AffinityPropagation(affinity="precomputed", damping=0.9, preference=p,
                                        max_iter=400, convergence_iter=400, random_state=0).fit(Sk)
        assert metrics.adjusted_rand_score(e, ap.labels_) == pytest.approx(1.0)


# ------------------------------------------------------------- brute force
def _brute_force(S):
    n = S.shape[0]
    best, best_e = -np.inf, None
    for r in range(1, n + 1):
        for E in itertools.combinations(range(n), r):
            e = np.array([i if i in E else max(E, key=lambda k: S[i, k]) for i in range(n)])
            v = sum(S[i, e[i]] for i in range(n))
            if v > best:
                best, best_e = v, e
    return best, best_e


def test_net_similarity_and_brute_force_optimum():
    optimal = consistent = 0
    total = 40
    for s in range(total):
        n, k = 6 + s % 5, 2 + s % 2
        X, _ = W.tiny_instance(n, k, 0.3, seed=s)
        S0 = H.neg_sq_euclidean(X)
        S = H.level_similarities(S0, [H.median_preference(S0)])
        best, best_e = _brute_force(S[0])
        # the objective of an assignment is the plain sum of its similarities
        assert H.net_similarity(S, best_e[None])[0] == pytest.approx(best, rel=1e-14)
        st = H.run(S, 500, 0.5, H.FIXED)
        e = H.exemplars(st.A, st.R)[0]
        if np.all(e[e] == e):
            consistent += 1
            ns = H.net_similarity(S, e[None])[0]
            # a valid configuration can never beat the exhaustive optimum
            assert ns <= best + 1e-12 * abs(best)
            optimal += ns >= best - 1e-12 * abs(best)
    assert consistent >= 0.95 * total
    assert optimal >= 0.70 * consistent


# ------------------------------------------------------------- invariants
def _random_problem(n=40, L=3, seed=3):
    X, _ = W.gmm_points(n, 2, 4, sigma=0.6, seed=seed)
    S0 = H.neg_sq_euclidean(X)
    p = H.median_preference(S0)
    prefs = np.array([p * (1.0 + 0.5 * l) for l in range(L)])
    return S0, prefs


@pytest.mark.parametrize("c_mode", [H.PAPER, H.FIXED])
@pytest.mark.parametrize("k", [-3, 5])
def test_power_of_two_scaling_is_exact(c_mode, k):
    S0, prefs = _random_problem()
    S = H.level_similarities(S0, prefs)
    a = H.run(S, 15, 0.6, c_mode)
    b = H.run(S * 2.0 ** k, 15, 0.6, c_mode)
    for fld in ("A", "R", "c", "tau", "phi"):
        np.testing.assert_array_equal(getattr(b, fld), getattr(a, fld) * 2.0 ** k, err_msg=fld)
    np.testing.assert_array_equal(H.exemplars(a.A, a.R), H.exemplars(b.A, b.R))


@pytest.mark.parametrize("c_mode", [H.PAPER, H.FIXED])
def test_permutation_equivariance(c_mode):
    S0, prefs = _random_problem(n=30, seed=5)
    perm = np.random.default_rng(1).permutation(S0.shape[0])
    S = H.level_similarities(S0, prefs)
    Sp = H.level_similarities(S0[np.ix_(perm, perm)], prefs)
    a = H.run(S, 12, 0.5, c_mode)
    b = H.run(Sp, 12, 0.5, c_mode)
    for fld in ("A", "R"):
        x = getattr(a, fld)[:, perm][:, :, perm]
        assert np.abs(getattr(b, fld) - x).max() <= 1e-12 * max(1.0, np.abs(x).max()), fld
    for fld in ("c", "tau", "phi"):
        x = getattr(a, fld)[:, perm]
        y = getattr(b, fld)
        fin = np.isfinite(x)
        np.testing.assert_array_equal(np.isfinite(y), fin)
        assert np.abs(y[fin] - x[fin]).max(initial=0.0) <= 1e-12 * max(1.0, np.abs(x[fin]).max(initial=0.0))
    inv = np.argsort(perm)
    np.testing.assert_array_equal(inv[H.exemplars(a.A, a.R)[:, perm]], H.exemplars(b.A, b.R))


def test_converged_assignment_is_self_consistent():
    X, _ = W.gmm_points(80, 2, 5, sigma=0.5, seed=7, means="uniform", mean_scale=10)
    S0 = H.neg_sq_euclidean(X)
    S = H.level_similarities(S0, [H.median_preference(S0)])
    st = H.run(S, 500, 0.9, H.FIXED)
    e = H.exemplars(st.A, st.R)[0]
    assert np.all(e[e] == e)
    # every exemplar chooses itself and its self-evidence is positive
    ex = np.unique(e)
    assert np.all(np.diagonal(st.A[0])[ex] + np.diagonal(st.R[0])[ex] > 0)


def test_first_iteration_closed_form():
    """At t = 1 (alpha = rho = 0, tau = +inf) Eq. 2.1 reduces to
    rho_ij = (1 - lam)(s_ij - max_{k != j} s_ik) at every level, and phi^l is
    the row maximum of S^{l+1} (Eq. 2.5 with alpha = 0)."""
    S0, prefs = _random_problem(n=25, seed=11)
    S = H.level_similarities(_asymmetric(S0, 11), prefs)
    lam = 0.3
    st = H.step(S, H.init_state(S.shape[0], S.shape[1]), lam, H.PAPER)
    n = S.shape[1]
    for l in range(S.shape[0]):
        for i in range(n):
            for j in range(n):
                others = [S[l, i, k] for k in range(n) if k != j]
                assert st.R[l, i, j] == pytest.approx((1 - lam) * (S[l, i, j] - max(others)), abs=1e-12)
        if l + 1 < S.shape[0]:
            np.testing.assert_array_equal(st.phi[l], S[l + 1].max(axis=1))
    assert np.all(st.phi[-1] == 0) and np.all(np.isinf(st.tau))


# ------------------------------------------------------------- library checks
def test_similarity_matches_scipy():
    from scipy.spatial.distance import cdist
    X, _ = W.gmm_points(50, 7, 3, sigma=1.0, seed=2)
    np.testing.assert_allclose(H.neg_sq_euclidean(X), -cdist(X, X, "sqeuclidean"), rtol=1e-13, atol=1e-12)
    np.testing.assert_allclose(H.neg_sq_euclidean_fixed_order(X, block=16), -cdist(X, X, "sqeuclidean"),
                               rtol=1e-13, atol=1e-12)


def test_fixed_order_similarity_is_exact_on_integers():
    """Small integer coordinates make every float64 operation exact, so the
    fixed-order sum must equal the integer definition -sum_k (x_ik - x_jk)^2
    computed with Python integers."""
    rng = np.random.default_rng(4)
    Xi = rng.integers(-50, 51, size=(37, 5))
    want = np.array([[-sum(int(a - b) ** 2 for a, b in zip(xi, xj)) for xj in Xi] for xi in Xi], dtype=np.float64)
    np.testing.assert_array_equal(H.neg_sq_euclidean_fixed_order(Xi.astype(np.float64), block=8), want)
    # the coordinate order is part of the definition: reversing it is a different rounding
    # sequence, but on exact inputs the same value
    np.testing.assert_array_equal(H.neg_sq_euclidean_fixed_order(Xi[:, ::-1].astype(np.float64)), want)


def test_adjusted_rand_index():
    rng = np.random.default_rng(0)
    a = rng.integers(0, 5, 200)
    assert H.adjusted_rand_index(a, a) == 1.0
    assert H.adjusted_rand_index(a, (a + 3) % 5) == 1.0  # relabelling
    # closed form for two labelings of 4 points: {0,0,1,1} vs {0,1,0,1} gives -0.5
    assert H.adjusted_rand_index([0, 0, 1, 1], [0, 1, 0, 1]) == pytest.approx(-0.5)
    metrics = pytest.importorskip("sklearn.metrics")
    b = rng.integers(0, 7, 200)
    assert H.adjusted_rand_index(a, b) == pytest.approx(metrics.adjusted_rand_score(a, b), abs=1e-12)


def test_exemplar_ties_take_lowest_index():
    """Eq. 2.8 with ties (reading R7): the lowest column index wins."""
    A = np.zeros((1, 3, 4))
    R = np.array([[[1.0, 3.0, 3.0, 0.0], [2.0, 2.0, 2.0, 2.0], [0.0, 0.0, 0.0, 5.0]]])
    np.testing.assert_array_equal(H.exemplars(A, R), [[1, 0, 3]])


def test_hierarchical_labels():
    e = np.array([[1, 1, 2, 2], [2, 1, 2, 2]])
    np.testing.assert_array_equal(H.hierarchical_labels(e), [[1, 1, 2, 2], [1, 1, 2, 2]])


def test_message_rel_error():
    x = np.array([[np.inf, 1.0], [2.0, -4.0]])
    assert H.message_rel_error(x, x) == 0.0
    y = x.copy()
    y[1, 1] = -4.004
    assert H.message_rel_error(y, x) == pytest.approx(1e-3)
    y = x.copy()
    y[0, 0] = 5.0
    assert H.message_rel_error(y, x) == float("inf")


def test_row_block_column_sums_partition():
    """Column sums over a partition of the rows add up to P_j of the whole
    matrix, and a hand-checked 3 x 3 case (negative entries and the diagonal
    drop out)."""
    R = np.array([[5.0, -1.0, 2.0], [3.0, 7.0, -4.0], [0.5, 1.5, 9.0]])
    assert np.array_equal(H.positive_column_sums(R), [3.5, 1.5, 2.0])
    assert np.array_equal(H.row_block_column_sums(R[1:], np.array([1, 2])), [3.5, 1.5, 0.0])
    rng = np.random.default_rng(4)
    R = rng.normal(size=(37, 37))
    parts = [np.arange(0, 10), np.arange(10, 11), np.arange(11, 37)]
    total = sum(H.row_block_column_sums(R[b], b) for b in parts)
    assert np.allclose(total, H.positive_column_sums(R), rtol=0, atol=1e-12)


# ------------------------------------------------ level schedule and Eq. 2.7
@pytest.mark.parametrize("c_mode", [H.PAPER, H.FIXED])
def test_one_level_gauss_seidel_equals_data_parallel(c_mode):
    """With one level there is no inter-level message, and c enters the
    availability update with the same value under both schedules (the row
    maximum of the previous iteration's A + R), so A and R agree exactly."""
    X, _ = W.gmm_points(12, 2, 3, sigma=0.5, seed=7, means="uniform", mean_scale=5.0)
    S = H.level_similarities(H.neg_sq_euclidean(X), [-8.0])
    a = H.init_state(1, 12)
    b = H.init_state(1, 12)
    for _ in range(25):
        a = H.step(S, a, 0.5, c_mode, H.JACOBI)
        b = H.step(S, b, 0.5, c_mode, H.GAUSS_SEIDEL)
        assert np.array_equal(a.A, b.A) and np.array_equal(a.R, b.R)


@pytest.mark.parametrize("schedule,kappa", [(H.GAUSS_SEIDEL, 0.0), (H.JACOBI, 0.25), (H.GAUSS_SEIDEL, 0.25)])
def test_variants_scale_exactly(schedule, kappa):
    """Power-of-two scaling of S scales every message bitwise under the
    sequential schedule and with Eq. 2.7 (kappa times a scaled sum)."""
    X, _ = W.gmm_points(15, 2, 3, sigma=0.5, seed=3, means="uniform", mean_scale=5.0)
    S = H.level_similarities(H.neg_sq_euclidean(X), [-6.0, -9.0, -12.0])
    a = H.run(S, 7, 0.5, H.PAPER, schedule=schedule, kappa=kappa)
    b = H.run(S * 8.0, 7, 0.5, H.PAPER, schedule=schedule, kappa=kappa)
    for f in ("A", "R", "c", "tau", "phi"):
        assert np.array_equal(getattr(a, f) * 8.0, getattr(b, f)), f


@pytest.mark.parametrize("schedule,kappa", [(H.GAUSS_SEIDEL, 0.0), (H.JACOBI, 0.25)])
def test_variants_permutation_equivariant(schedule, kappa):
    X, _ = W.gmm_points(14, 2, 3, sigma=0.5, seed=9, means="uniform", mean_scale=5.0)
    S = H.level_similarities(H.neg_sq_euclidean(X), [-6.0, -9.0])
    perm = np.random.default_rng(2).permutation(14)
    a = H.run(S, 6, 0.5, H.PAPER, schedule=schedule, kappa=kappa)
    b = H.run(S[:, perm][:, :, perm], 6, 0.5, H.PAPER, schedule=schedule, kappa=kappa)
    np.testing.assert_allclose(a.A[:, perm][:, :, perm], b.A, rtol=0, atol=1e-12)
    np.testing.assert_allclose(a.R[:, perm][:, :, perm], b.R, rtol=0, atol=1e-12)


def test_purity():
    """Purity (§4): hand example and its extreme cases."""
    assert H.purity([0, 0, 1, 1, 1], ["a", "a", "a", "b", "b"]) == 4 / 5
    truth = np.array([0, 0, 1, 2, 2, 2])
    assert H.purity(truth, truth) == 1.0
    assert H.purity(np.arange(6), truth) == 1.0
    assert H.purity(np.zeros(6), truth) == 3 / 6
    assert H.purity(np.array([5, 5, 5, 7, 7, 7]), truth) == (2 + 3) / 6


def test_acceptance_counts():
    """Hand examples: [1, 1, 2, 1] is self-consistent with exemplars 1 and 2;
    in [1, 2, 2, 0] points 0 and 3 point at non-exemplars."""
    cons, ex = H.acceptance(np.array([[1, 1, 2, 1], [1, 2, 2, 0]]))
    assert list(cons) == [4, 2] and list(ex) == [2, 1]
