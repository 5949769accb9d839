"""FP64 reference implementation ("oracle") of Hierarchical Affinity Propagation.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this module:
only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference leg of ``bench.py`` may use it.  It shares no code with the CUDA
library; the two meet only through arrays.

Source: D. M. Rose, J. M. Rouly, R. Haber, N. Mijatovic, A. M. Peter,
"Parallel Hierarchical Affinity Propagation with MapReduce" (arXiv:1403.7394):
  * §2, Eq. 2.1  responsibility      rho_ij^l
  * §2, Eq. 2.2  availability        alpha_ij^l   (i != j)
  * §2, Eq. 2.3  self-availability   alpha_jj^l
  * §2           damping by lambda of rho and alpha at every level
  * §2, Eq. 2.4  bottom-up message   tau_j^{l+1}
  * §2, Eq. 2.5  top-down message    phi_i^{l-1}
  * §2, Eq. 2.6  cluster preference  c_i^l
  * §2, Eq. 2.8  exemplar assignment e_i^l
  * §2, Algorithm 1 (initial values, iteration structure)
  * §3 (MR-HAP jobs): tau and c are not updated in the first iteration, and
    every (i, l) is updated in one job from the start-of-iteration state.

Everything is float64 and written for clarity, not speed: each function is one
equation, whole rows or whole matrices at a time, with numpy reductions as the
only library primitives.

Index conventions: levels are 0-based here (the paper's level l is index l-1);
for the (L, N, N) tensors S, A (alpha) and R (rho) axis 1 is the node i and
axis 2 the candidate exemplar j (the paper's §3 tensor layout); c, tau and phi
are (L, N).

Readings of points the paper leaves open (each is also listed in the design
notes of the repository):
  R1  Damping: m <- lam * m_old + (1 - lam) * m_new.
  R2  Eq. 2.6 is a row maximum that includes j = i; its result is used as c_j
      in Eqs. 2.2-2.4 for node j.
  R3  Boundary levels: tau at the lowest level is +inf (Eq. 2.1 is stated for
      l > 1 and Algorithm 1 starts tau at infinity); phi at the top level is 0
      (Eq. 2.2 is stated for l < L and Algorithm 1 starts phi at 0).
  R4  Level schedule "jacobi" (the data-parallel MR-HAP schedule of §3): every
      inter-level quantity of iteration t is computed from the state at the
      start of t; tau^{l} uses c^{l-1} computed in the same iteration.
  R5  Iteration 1 computes neither c nor tau (§3); phi is computed from t = 1.
  R6  Within an iteration rho is updated first, then alpha from the new, damped
      rho (Algorithm 1).
  R7  max_{k != j} excludes only index j; ties keep the lowest index for the
      argmax in Eq. 2.5's rho use and in Eq. 2.8.
  R8  c_mode "paper" applies Eq. 2.6 each iteration from t = 2; c_mode "fixed"
      keeps c at its initial value (0 unless given), which makes L = 1
      identical to flat affinity propagation.
  R9  Net similarity, not defined in the paper, is NS^l = sum_i s^l_{i, e_i^l}
      with s^l_ii the preference of level l.
  R10 Eq. 2.7 (optional level-wise similarity update; its index j is both
      free and bound as printed) is read element-wise:
      s^{l+1}_ij = s^l_ij + kappa (alpha^l_ij + rho^l_ij) for i != j, the
      diagonal of level l+1 staying its preference.  kappa = 0 (default)
      leaves every level's S as given.  Jacobi: built from the
      start-of-iteration messages; Gauss-Seidel: from level l's messages just
      updated.  NS (R9) keeps using the given S.
  R11 Level schedule "gauss_seidel" (Algorithm 1's sequential level loop):
      for l = 1..L in order, rho^l (Eq. 2.1 with the tau^l that level l-1
      sent in this iteration, +inf at l = 1), then alpha^l (Eqs. 2.2-2.3 with
      c^l and phi^l as they stand), then the messages level l sends: c^l
      (Eq. 2.6, c_mode "paper"), tau^{l+1} (Eq. 2.4) and phi^{l-1} (Eq. 2.5)
      from the new alpha^l and rho^l.  Algorithm 1 has no first-iteration
      exception, so c and tau are updated from t = 1; phi starts at 0.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

PAPER = "paper"
FIXED = "fixed"
JACOBI = "jacobi"
GAUSS_SEIDEL = "gauss_seidel"


# ---------------------------------------------------------------------------
# Inputs: similarities and preferences (§2)
# ---------------------------------------------------------------------------
def neg_sq_euclidean(X, rows=None) -> np.ndarray:
    """s_ij = -||x_i - x_j||^2 in float64, straight from the definition (§2:
    the negative squared Euclidean distance is the usual similarity).  The
    diagonal is 0 here; preferences are placed on it separately.  ``rows``
    selects the rows i to compute (all by default)."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    rows = np.arange(n) if rows is None else np.asarray(rows)
    S = np.empty((rows.size, n), dtype=np.float64)
    for r, i in enumerate(rows):
        d = X - X[i]
        S[r] = -np.einsum("kd,kd->k", d, d)
    return S


def neg_sq_euclidean_fixed_order(X, block: int = 512, rows=None) -> np.ndarray:
    """The same similarity as ``neg_sq_euclidean`` (§2), with the sum over the
    coordinates taken in order k = 0, 1, ..., d-1, one correctly rounded
    float64 subtraction, multiplication and addition at a time.  Every
    IEEE-754 machine then produces the same bits, so a similarity built on
    one host can be rebuilt bit for bit on another (a library reduction may
    change its summation order between builds).  ``rows`` selects the rows i
    to compute (all by default)."""
    X = np.asarray(X, dtype=np.float64)
    n, d = X.shape
    rows = np.arange(n) if rows is None else np.asarray(rows)
    S = np.empty((rows.size, n), dtype=np.float64)
    for r0 in range(0, rows.size, block):
        r1 = min(rows.size, r0 + block)
        acc = np.zeros((r1 - r0, n), dtype=np.float64)
        for k in range(d):
            diff = np.subtract.outer(X[rows[r0:r1], k], X[:, k])
            acc += diff * diff
        S[r0:r1] = -acc
    return S


def median_preference(S) -> float:
    """Median of the off-diagonal entries of S, in float64 (a common choice of
    uniform preference; §2 lists uniform prior-knowledge settings)."""
    S = np.asarray(S, dtype=np.float64)
    n = S.shape[0]
    off = S[~np.eye(n, dtype=bool)]
    return float(np.median(off))


def level_similarities(S, prefs) -> np.ndarray:
    """The (L, N, N) similarity tensor of §3 when every level shares the same
    off-diagonal similarities: level l is S with its diagonal (the
    preferences s_jj, §2) set to prefs[l] (a scalar or a length-N vector)."""
    S = np.asarray(S, dtype=np.float64)
    prefs = np.asarray(prefs, dtype=np.float64)
    L = prefs.shape[0]
    n = S.shape[0]
    out = np.empty((L, n, n), dtype=np.float64)
    idx = np.arange(n)
    for l in range(L):
        out[l] = S
        out[l, idx, idx] = prefs[l]
    return out


# ---------------------------------------------------------------------------
# Message updates (§2)
# ---------------------------------------------------------------------------
def damp(old, new, lam):
    """Damping of a message by lambda (§2): lam * old + (1 - lam) * new."""
    return lam * old + (1.0 - lam) * new


def responsibility_update(S_rows, A_rows, R_rows, tau_rows, lam):
    """Eq. 2.1 with damping, for a block of whole rows of one level.

    rho_ij <- s_ij + min(tau_i, -max_{k != j}(alpha_ik + s_ik)).
    The maximum over k != j equals the row maximum m1 except in the column k1
    that attains it (lowest index on ties), where it is the second largest
    value m2 (which equals m1 when the maximum is attained twice)."""
    X = A_rows + S_rows
    rows = np.arange(X.shape[0])
    k1 = np.argmax(X, axis=1)  # first occurrence: lowest index
    m1 = X[rows, k1]
    X_wo = X.copy()
    X_wo[rows, k1] = -np.inf
    m2 = np.max(X_wo, axis=1)
    max_excl = np.repeat(m1[:, None], X.shape[1], axis=1)
    max_excl[rows, k1] = m2
    R_hat = S_rows + np.minimum(np.asarray(tau_rows, dtype=np.float64)[:, None], -max_excl)
    return damp(R_rows, R_hat, lam)


def positive_column_sums(R_l, partition=None) -> np.ndarray:
    """P_j = sum_{k != j} max(0, rho_kj): the evidence sum shared by Eqs. 2.2,
    2.3 and 2.4, for one level.

    ``partition`` (a list of row-index arrays covering every row once) only
    fixes the order of the float64 sum: each part's rows are summed by
    ``row_block_column_sums`` and the part sums are added in list order -
    the order in which a row-sharded run combines its shards."""
    if partition is not None:
        P = None
        for rows in partition:
            part = row_block_column_sums(R_l[np.asarray(rows)], rows)
            P = part if P is None else P + part
        return P
    Rp = np.maximum(R_l, 0.0)
    n = R_l.shape[0]
    Rp[np.arange(n), np.arange(n)] = 0.0
    return Rp.sum(axis=0)


def row_block_column_sums(R_rows, rows) -> np.ndarray:
    """The part of P_j (positive_column_sums) contributed by the whole rows
    ``rows`` of one level: sum over k in rows, k != j, of max(0, rho_kj).
    Summing it over a partition of the rows gives P_j."""
    rows = np.asarray(rows)
    Rp = np.maximum(R_rows, 0.0)
    Rp[np.arange(rows.size), rows] = 0.0
    return Rp.sum(axis=0)


def availability_update(A_rows, R_rows, rows, c_l, phi_l, R_diag, P, lam):
    """Eqs. 2.2 and 2.3 with damping, for the rows ``rows`` of one level.

    R_rows are the (already updated) responsibilities of those rows, R_diag
    and P the diagonal and positive column sums of the full updated
    responsibility matrix of the level (Eq. 2.2's sum over k not in {i, j}
    is P_j minus the k = i term).
        alpha_ij <- min(0, c_j + phi_j + rho_jj + P_j - max(0, rho_ij))  (i != j)
        alpha_jj <- c_j + phi_j + P_j
    """
    rows = np.asarray(rows)
    base = c_l + phi_l + R_diag + P  # c_j + phi_j + rho_jj + P_j, per column j
    A_hat = np.minimum(0.0, base[None, :] - np.maximum(0.0, R_rows))
    r = np.arange(rows.shape[0])
    A_hat[r, rows] = (c_l + phi_l + P)[rows]
    return damp(A_rows, A_hat, lam)


def tau_update(c, R, partition=None) -> np.ndarray:
    """Eq. 2.4: tau_j^{l+1} = c_j^l + rho_jj^l + sum_{k != j} max(0, rho_kj^l);
    the lowest level has tau = +inf (reading R3)."""
    L, n, _ = R.shape
    tau = np.full((L, n), np.inf)
    for l in range(1, L):
        tau[l] = c[l - 1] + np.diagonal(R[l - 1]) + positive_column_sums(R[l - 1], partition)
    return tau


def phi_update(A, S) -> np.ndarray:
    """Eq. 2.5: phi_i^{l-1} = max_k (alpha_ik^l + s_ik^l); the top level has
    phi = 0 (reading R3)."""
    L, n, _ = A.shape
    phi = np.zeros((L, n))
    for l in range(L - 1):
        phi[l] = np.max(A[l + 1] + S[l + 1], axis=1)
    return phi


def cluster_preference_update(A, R) -> np.ndarray:
    """Eq. 2.6: c_i^l = max_j (alpha_ij^l + rho_ij^l)."""
    return np.max(A + R, axis=2)


# ---------------------------------------------------------------------------
# State and iteration (Algorithm 1, §3 schedule)
# ---------------------------------------------------------------------------
@dataclass
class HAPState:
    """Messages after ``t`` completed iterations (Algorithm 1 initial values
    at t = 0: alpha = rho = 0, tau = +inf, phi = 0, c = c0 (0 by default))."""

    A: np.ndarray
    R: np.ndarray
    c: np.ndarray
    tau: np.ndarray
    phi: np.ndarray
    t: int = 0
    extra: dict = field(default_factory=dict)

    def copy(self) -> "HAPState":
        return HAPState(self.A.copy(), self.R.copy(), self.c.copy(),
                        self.tau.copy(), self.phi.copy(), self.t)


def init_state(L: int, N: int, c0=None) -> HAPState:
    c = np.zeros((L, N)) if c0 is None else np.array(c0, dtype=np.float64).reshape(L, N)
    return HAPState(A=np.zeros((L, N, N)), R=np.zeros((L, N, N)), c=c,
                    tau=np.full((L, N), np.inf), phi=np.zeros((L, N)), t=0)


def similarity_level_update(S_l, A_l, R_l, pref_next, kappa):
    """Eq. 2.7 (reading R10): the level-(l+1) similarity from level l,
    s_ij + kappa (alpha_ij + rho_ij) off the diagonal, pref_next on it."""
    out = S_l + kappa * (A_l + R_l)
    idx = np.arange(S_l.shape[0])
    out[idx, idx] = pref_next
    return out


def step(S, st: HAPState, lam: float, c_mode: str = PAPER, schedule: str = JACOBI,
         kappa: float = 0.0, partition=None) -> HAPState:
    """One HAP iteration (number st.t + 1) on the (L, N, N) similarity tensor S.

    Order (readings R4-R6): inter-level quantities from the start-of-iteration
    state, then rho at every level (Eq. 2.1), then alpha at every level from
    the new rho (Eqs. 2.2-2.3).  schedule="gauss_seidel" runs Algorithm 1's
    level loop instead (R11); kappa > 0 applies Eq. 2.7 (R10).  ``partition``
    fixes the summation order of the column sums (positive_column_sums)."""
    if schedule == GAUSS_SEIDEL:
        return step_gauss_seidel(S, st, lam, c_mode, kappa)
    if schedule != JACOBI:
        raise ValueError(f"unknown schedule {schedule!r}")
    S = np.asarray(S, dtype=np.float64)
    L, n, _ = S.shape
    if kappa:
        S = S.copy()
        for l in range(L - 1):                                 # Eq. 2.7
            S[l + 1] = similarity_level_update(S[l], st.A[l], st.R[l], np.diagonal(S[l + 1]), kappa)
    t = st.t + 1
    c = st.c.copy()
    if t >= 2:
        if c_mode == PAPER:
            c = cluster_preference_update(st.A, st.R)          # Eq. 2.6
        tau = tau_update(c, st.R, partition)                   # Eq. 2.4
    else:
        tau = np.full((L, n), np.inf)
    phi = phi_update(st.A, S)                                  # Eq. 2.5

    R_new = np.empty_like(st.R)
    for l in range(L):                                         # Eq. 2.1
        R_new[l] = responsibility_update(S[l], st.A[l], st.R[l], tau[l], lam)

    A_new = np.empty_like(st.A)
    rows = np.arange(n)
    for l in range(L):                                         # Eqs. 2.2, 2.3
        P = positive_column_sums(R_new[l], partition)
        A_new[l] = availability_update(st.A[l], R_new[l], rows, c[l], phi[l],
                                       np.diagonal(R_new[l]).copy(), P, lam)
    return HAPState(A=A_new, R=R_new, c=c, tau=tau, phi=phi, t=t)


def step_gauss_seidel(S, st: HAPState, lam: float, c_mode: str = PAPER, kappa: float = 0.0) -> HAPState:
    """One iteration of Algorithm 1's sequential level loop (reading R11):
    level by level, rho^l, then alpha^l, then the messages level l sends
    (c^l, tau^{l+1}, phi^{l-1}) and, with kappa > 0, the level-(l+1)
    similarity (Eq. 2.7)."""
    S = np.array(S, dtype=np.float64)
    L, n, _ = S.shape
    A, R, c, phi = st.A.copy(), st.R.copy(), st.c.copy(), st.phi.copy()
    tau = np.full((L, n), np.inf)
    rows = np.arange(n)
    for l in range(L):
        R[l] = responsibility_update(S[l], A[l], R[l], tau[l], lam)                  # Eq. 2.1
        P = positive_column_sums(R[l])
        Rd = np.diagonal(R[l]).copy()
        A[l] = availability_update(A[l], R[l], rows, c[l], phi[l], Rd, P, lam)        # Eqs. 2.2, 2.3
        if c_mode == PAPER:
            c[l] = cluster_preference_update(A[l][None], R[l][None])[0]               # Eq. 2.6
        if l + 1 < L:
            tau[l + 1] = c[l] + Rd + P                                               # Eq. 2.4
            if kappa:
                S[l + 1] = similarity_level_update(S[l], A[l], R[l], np.diagonal(S[l + 1]), kappa)  # Eq. 2.7
        if l >= 1:
            phi[l - 1] = phi_update(np.stack([A[l], A[l]]), np.stack([S[l], S[l]]))[0]  # Eq. 2.5
    return HAPState(A=A, R=R, c=c, tau=tau, phi=phi, t=st.t + 1)


def run(S, iterations: int, lam: float, c_mode: str = PAPER, c0=None,
        state: HAPState | None = None, callback=None, schedule: str = JACOBI,
        kappa: float = 0.0, partition=None) -> HAPState:
    """Algorithm 1's iteration loop for a fixed number of iterations."""
    S = np.asarray(S, dtype=np.float64)
    L, n, _ = S.shape
    st = init_state(L, n, c0) if state is None else state
    for _ in range(iterations):
        st = step(S, st, lam, c_mode, schedule, kappa, partition)
        if callback is not None:
            callback(st)
    return st


def level_similarity_rows(S_rows, rows, prefs) -> np.ndarray:
    """The whole rows ``rows`` of the (L, N, N) similarity tensor of
    ``level_similarities``: S_rows (len(rows), N) are rows of the shared
    off-diagonal similarities; level l puts prefs[l] on the diagonal entries
    (i, i) of its owned rows i."""
    S_rows = np.asarray(S_rows, dtype=np.float64)
    rows = np.asarray(rows)
    prefs = np.asarray(prefs, dtype=np.float64)
    L = prefs.shape[0]
    out = np.empty((L,) + S_rows.shape, dtype=np.float64)
    loc = np.arange(rows.size)
    for l in range(L):
        out[l] = S_rows
        out[l, loc, rows] = prefs[l] if prefs.ndim == 1 else prefs[l, rows]
    return out


def init_shard_state(L: int, N: int, rows, c0=None) -> HAPState:
    """Algorithm 1's initial values for the shard that owns ``rows``: alpha
    and rho (L, len(rows), N) zero; the vectors c, tau, phi keep all N
    nodes."""
    nr = np.asarray(rows).size
    c = np.zeros((L, N)) if c0 is None else np.array(c0, dtype=np.float64).reshape(L, N)
    return HAPState(A=np.zeros((L, nr, N)), R=np.zeros((L, nr, N)), c=c,
                    tau=np.full((L, N), np.inf), phi=np.zeros((L, N)), t=0)


def step_sharded(S_rows, st: HAPState, rows, lam: float, c_mode: str, allreduce,
                 carry: dict | None = None):
    """One iteration of ``step`` computed by the shard that owns the whole rows
    ``rows`` of a row-partitioned problem (MR-HAP, §3, keys its messages by
    node; here a shard is a band of nodes).  The shard holds only its rows:
    S_rows, st.A and st.R are (L, len(rows), N); the vectors c, tau and phi
    are (L, N).  Every row quantity (rho, alpha, c, tau, phi of node i) is
    computed for owned rows only, and everything another shard needs - the
    positive column sums and the owned diagonal, c and phi values (zero
    elsewhere) - crosses shards through ONE sum all-reduce per iteration
    (``allreduce(x)`` returns the element-wise sum of x over all shards).

    ``carry`` holds the previous iteration's reduced column statistics of rho
    ({"P": (L, N), "Rdiag": (L, N)}); None at the first iteration of a run
    (or after a restart, when they are recomputed with one extra reduction).
    With the shards' partial sums added in shard order, the result has the
    bits of ``step(..., partition=<the shards' rows in order>)``."""
    S_rows = np.asarray(S_rows, dtype=np.float64)
    L, nr, n = S_rows.shape
    rows = np.asarray(rows)
    loc = np.arange(nr)
    t = st.t + 1
    A, R = st.A, st.R
    if carry is None:  # column statistics of the current rho (Eqs. 2.2-2.4 sums)
        part = np.zeros((2, L, n))
        for l in range(L):
            part[0, l] = row_block_column_sums(R[l], rows)
            part[1, l, rows] = R[l][loc, rows]
        part = allreduce(part)
        carry = {"P": part[0], "Rdiag": part[1]}
    c = st.c.copy()
    if t >= 2 and c_mode == PAPER:                              # Eq. 2.6, owned rows
        c[:, rows] = np.max(A + R, axis=2)
    tau = np.full((L, n), np.inf)
    if t >= 2:                                                  # Eq. 2.4, owned rows
        for l in range(1, L):
            tau[l, rows] = c[l - 1, rows] + carry["Rdiag"][l - 1, rows] + carry["P"][l - 1, rows]
    phi = np.zeros((L, n))
    for l in range(L - 1):                                      # Eq. 2.5, owned rows
        phi[l, rows] = np.max(A[l + 1] + S_rows[l + 1], axis=1)
    R_new = np.empty_like(R)
    for l in range(L):                                          # Eq. 2.1, owned rows
        R_new[l] = responsibility_update(S_rows[l], A[l], R[l], tau[l, rows], lam)
    # the one exchange: column sums of the new rho, and the owned c, phi, rho_jj
    part = np.zeros((4, L, n))
    for l in range(L):
        part[0, l] = row_block_column_sums(R_new[l], rows)
        part[1, l, rows] = R_new[l][loc, rows]
        part[2, l, rows] = c[l, rows]
        part[3, l, rows] = phi[l, rows]
    part = allreduce(part)
    A_new = np.empty_like(A)
    for l in range(L):                                          # Eqs. 2.2, 2.3, owned rows
        A_new[l] = availability_update(A[l], R_new[l], rows, part[2, l], part[3, l], part[1, l], part[0, l], lam)
    out = HAPState(A=A_new, R=R_new, c=part[2], tau=tau, phi=part[3], t=t)
    return out, {"P": part[0], "Rdiag": part[1]}


# ---------------------------------------------------------------------------
# Outputs (Eq. 2.8) and the objective
# ---------------------------------------------------------------------------
def exemplars(A, R) -> np.ndarray:
    """Eq. 2.8: e_i^l = argmax_j (alpha_ij^l + rho_ij^l), lowest index on
    ties; returns int32 (L, N)."""
    return np.argmax(np.asarray(A) + np.asarray(R), axis=2).astype(np.int32)


def net_similarity(S, e) -> np.ndarray:
    """NS^l = sum_i s^l_{i, e_i^l} in float64 (reading R9); S is (L, N, N)
    with the preferences on the diagonal."""
    S = np.asarray(S, dtype=np.float64)
    e = np.asarray(e)
    L, n, _ = S.shape
    return np.array([S[l, np.arange(n), e[l]].sum() for l in range(L)])


def hierarchical_labels(e) -> np.ndarray:
    """Chains the per-level assignments: h^0(i) = e^0_i and
    h^l(i) = e^l_{h^{l-1}(i)}, giving every point a label at every level."""
    e = np.asarray(e)
    L, n = e.shape
    h = np.empty_like(e)
    h[0] = e[0]
    for l in range(1, L):
        h[l] = e[l][h[l - 1]]
    return h


def adjusted_rand_index(a, b) -> float:
    """Adjusted Rand index (Hubert & Arabie 1985) of two labelings, from the
    contingency table, in float64."""
    a = np.asarray(a)
    b = np.asarray(b)
    _, ai = np.unique(a, return_inverse=True)
    _, bi = np.unique(b, return_inverse=True)
    table = np.zeros((ai.max() + 1, bi.max() + 1), dtype=np.float64)
    np.add.at(table, (ai, bi), 1.0)

    def comb2(x):
        return x * (x - 1.0) / 2.0

    n = float(a.shape[0])
    sum_ij = comb2(table).sum()
    sum_a = comb2(table.sum(axis=1)).sum()
    sum_b = comb2(table.sum(axis=0)).sum()
    expected = sum_a * sum_b / comb2(n) if n > 1 else 0.0
    max_index = 0.5 * (sum_a + sum_b)
    if max_index == expected:
        return 1.0
    return float((sum_ij - expected) / (max_index - expected))


def acceptance(e):
    """Acceptance check of an assignment (Eq. 2.8), per level: the number of
    points whose exemplar is its own exemplar (e[e_i] == e_i) and the number
    of exemplars (e_i == i)."""
    e = np.atleast_2d(np.asarray(e))
    idx = np.arange(e.shape[1])
    cons = np.array([int(np.sum(el[el] == el)) for el in e])
    ex = np.array([int(np.sum(el == idx)) for el in e])
    return cons, ex


def purity(labels, truth) -> float:
    """Purity, the extrinsic cluster-quality measure of §4: the fraction of
    points that carry the most frequent true class of their cluster,
    (1/N) sum over clusters of max over classes |cluster and class|."""
    labels = np.asarray(labels).ravel()
    truth = np.asarray(truth).ravel()
    total = 0
    for k in np.unique(labels):
        _, counts = np.unique(truth[labels == k], return_counts=True)
        total += int(counts.max())
    return total / labels.size


def message_rel_error(x_test, x_ref) -> float:
    """max |x_test - x_ref| / max(max |x_ref|, 1) over the finite entries of
    x_ref; infinite entries must match exactly (used for tau)."""
    x_test = np.asarray(x_test, dtype=np.float64)
    x_ref = np.asarray(x_ref, dtype=np.float64)
    fin = np.isfinite(x_ref)
    if not np.array_equal(np.isfinite(x_test), fin):
        return float("inf")
    if not np.array_equal(x_test[~fin], x_ref[~fin]):
        return float("inf")
    if not fin.any():
        return 0.0
    scale = max(float(np.max(np.abs(x_ref[fin]))), 1.0)
    return float(np.max(np.abs(x_test[fin] - x_ref[fin])) / scale)
