"""Python binding of libhap (ctypes over the C ABI in include/hap.h).

Argument marshalling only: every step of the method runs in the CUDA library.
PyTorch supplies device memory (the workspace and the caller's tensors) and
the CUDA stream.  Importing this module loads libhap.so and raises if it is
missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhap.so")

HAP_OK, HAP_EINVAL, HAP_ENOMEM, HAP_ECUDA, HAP_EDEVICE, HAP_ETIMEOUT, HAP_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
C_MODES = {"paper": 0, "fixed": 1}
S_DTYPES = {"f32": 0, "bf16": 1}
SBUILD = {"f32": 0, "bf16": 1, "bf16_split": 2}
Q_BLOCK_THREADS, Q_CLUSTER_SIZE, Q_GRID_CLUSTERS, Q_LD, Q_ITER, Q_ELEMS_PER_THREAD, Q_LAUNCHES = 1, 2, 3, 4, 5, 6, 7
Q_BATCH_ITEMS_PER_CTA = 8
Q_COL_SUMS, Q_STAGES, Q_CTAS_PER_SM = 9, 10, 11
COL_SUMS = {"auto": 0, "smem": 1, "tmem": 2}
SCHEDULES = {"jacobi": 0, "gauss_seidel": 1}


class HapOptions(ctypes.Structure):
    _fields_ = [("c_mode", ctypes.c_int), ("schedule", ctypes.c_int), ("s_dtype", ctypes.c_int),
                ("s_per_level", ctypes.c_int), ("block_threads", ctypes.c_int),
                ("cluster_size", ctypes.c_int), ("grid_clusters", ctypes.c_int),
                ("elems_per_thread", ctypes.c_int), ("profile", ctypes.c_int), ("col_sums", ctypes.c_int),
                ("kappa", ctypes.c_float), ("wait_limit_ns", ctypes.c_int64), ("ctas_per_sm", ctypes.c_int),
                ("debug_bounds", ctypes.c_int)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1403_7394_gb300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, i32, f32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_float
    sigs = {
        "hap_default_options": (None, [ctypes.POINTER(HapOptions)]),
        "hap_workspace_bytes": (i32, [i64, i32, ctypes.POINTER(HapOptions), ctypes.POINTER(ctypes.c_size_t)]),
        "hap_create": (i32, [i64, i32, vp, f32, ctypes.POINTER(HapOptions), vp, ctypes.c_size_t, ctypes.POINTER(vp)]),
        "hap_destroy": (None, [vp]),
        "hap_set_stream": (i32, [vp, vp]),
        "hap_set_preferences": (i32, [vp, vp, i32]),
        "hap_set_cluster_preferences": (i32, [vp, vp]),
        "hap_set_similarity": (i32, [vp, i32, vp, i64, i32]),
        "hap_build_similarity": (i32, [vp, vp, i64, i32]),
        "hap_get_similarity": (i32, [vp, i32, vp]),
        "hap_iterate": (i32, [vp, i32]),
        "hap_exemplars": (i32, [vp, vp, i32]),
        "hap_net_similarity": (i32, [vp, vp]),
        "hap_get_state": (i32, [vp, vp, vp, vp, ctypes.POINTER(i64)]),
        "hap_set_state": (i32, [vp, vp, vp, vp, i64]),
        "hap_sync": (i32, [vp]),
        "hap_set_wait_limit": (i32, [vp, i64]),
        "hap_query": (i32, [vp, i32, ctypes.POINTER(i64)]),
        "hap_row_pass_time": (i32, [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64), i32]),
        "hap_strerror": (ctypes.c_char_p, [i32]),
        "hap_iterate_noalloc": (i32, [i64, i32, f32, i32, vp, i32, vp, vp, vp, vp, vp, vp, i64, i32, vp]),
        "hap_batch_create": (i32, [i32, vp, vp, f32, ctypes.POINTER(HapOptions), ctypes.POINTER(vp)]),
        "hap_batch_destroy": (None, [vp]),
        "hap_batch_set_stream": (i32, [vp, vp]),
        "hap_batch_set_preferences": (i32, [vp, vp]),
        "hap_batch_build_similarity": (i32, [vp, vp, i64, i32]),
        "hap_batch_set_similarity": (i32, [vp, i32, vp, i64, i32]),
        "hap_batch_iterate": (i32, [vp, i32]),
        "hap_batch_exemplars": (i32, [vp, vp, i32]),
        "hap_batch_net_similarity": (i32, [vp, vp]),
        "hap_batch_get_state": (i32, [vp, i32, vp, vp, vp, ctypes.POINTER(i64)]),
        "hap_batch_tune": (i32, [vp, ctypes.POINTER(ctypes.c_double)]),
        "hap_batch_set_tile": (i32, [vp, i32]),
        "hap_batch_set_wait_limit": (i32, [vp, i64]),
        "hap_batch_query": (i32, [vp, i32, ctypes.POINTER(i64)]),
        "hap_batch_sync": (i32, [vp]),
        "hap_knn": (i32, [vp, i64, i64, i32, vp, vp, vp]),
        "hap_acceptance": (i32, [vp, vp, vp]),
        "hap_knn_with": (i32, [vp, i64, i64, i32, i32, vp, vp, vp]),
        "hap_proposal_launches": (i64, []),
        "hap_knn_subset_with": (i32, [vp, i64, i64, vp, i64, i32, i32, vp, vp, vp]),
        "hap_knn_features": (i32, [vp, i64, i32, i32, vp, ctypes.POINTER(f32), vp]),
        "hap_knn_subset": (i32, [vp, i64, i64, vp, i64, i32, vp, vp, vp]),
        "hap_top_scores": (i32, [vp, i64, i64, vp, vp]),
        "hap_select_hub_candidates": (i32, [vp, i64, i32, vp, i32, i32, i32, vp, vp]),
        "hap_exemplar_points": (i32, [vp, i64, i64, vp, ctypes.POINTER(i64), vp]),
        "hap_mlp_create": (i32, [i32, vp, ctypes.POINTER(vp)]),
        "hap_mlp_destroy": (None, [vp]),
        "hap_mlp_set_stream": (i32, [vp, vp]),
        "hap_mlp_num_params": (i32, [vp, ctypes.POINTER(i64)]),
        "hap_mlp_get_params": (i32, [vp, vp]),
        "hap_mlp_forward": (i32, [vp, vp, i64, vp]),
        "hap_mlp_gradients": (i32, [vp, vp, vp, i64, f32, vp, vp]),
        "hap_mlp_train_step": (i32, [vp, vp, vp, i64, f32, f32, vp]),
        "hap_select_candidates": (i32, [vp, i64, i32, vp, i32, i32, vp, vp]),
        "hap_sparse_create": (i32, [i64, i32, i32, vp, f32, i32, ctypes.POINTER(vp)]),
        "hap_sparse_destroy": (None, [vp]),
        "hap_sparse_set_stream": (i32, [vp, vp]),
        "hap_sparse_set_preferences": (i32, [vp, vp, i32]),
        "hap_sparse_set_candidates": (i32, [vp, vp, vp, i64]),
        "hap_sparse_iterate": (i32, [vp, i32]),
        "hap_sparse_exemplars": (i32, [vp, vp, i32]),
        "hap_sparse_net_similarity": (i32, [vp, vp]),
        "hap_sparse_get_state": (i32, [vp, vp, vp, vp, ctypes.POINTER(i64)]),
        "hap_sparse_query": (i32, [vp, i32, ctypes.POINTER(i64)]),
        "hap_sparse_set_profile": (i32, [vp, i32]),
        "hap_sparse_profile_times": (i32, [vp, vp, ctypes.POINTER(i64), i32]),
        "hap_net_similarity_points": (i32, [vp, i64, i64, i32, vp, vp, vp, vp]),
        "hap_noalloc_scratch_bytes": (ctypes.c_size_t, []),
        "hap_band_create": (i32, [i64, i64, i64, i32, vp, f32, ctypes.POINTER(HapOptions), ctypes.POINTER(vp)]),
        "hap_band_destroy": (None, [vp]),
        "hap_band_set_stream": (i32, [vp, vp]),
        "hap_band_set_similarity": (i32, [vp, vp, i64, i32]),
        "hap_band_exchange_floats": (i32, [vp, ctypes.POINTER(i64)]),
        "hap_band_rows": (i32, [vp, vp]),
        "hap_band_columns": (i32, [vp, vp, i32, vp]),
        "hap_band_get_state": (i32, [vp, vp, vp, vp, ctypes.POINTER(i64)]),
        "hap_band_exemplars": (i32, [vp, vp, i32]),
        "hap_band_sync": (i32, [vp]),
        "hap_band_query": (i32, [vp, i32, ctypes.POINTER(i64)]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


class HapError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {lib.hap_strerror(code).decode()} ({code})")
        self.code = code


def check(code: int, what: str) -> None:
    if code != HAP_OK:
        raise HapError(code, what)


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def options(c_mode="paper", s_dtype="f32", s_per_level=False, block_threads=0, cluster_size=0,
            grid_clusters=0, elems_per_thread=0, profile=False, col_sums="auto", schedule="jacobi",
            kappa=0.0, wait_limit_ns=0, ctas_per_sm=0, debug_bounds=False) -> HapOptions:
    o = HapOptions()
    lib.hap_default_options(ctypes.byref(o))
    o.c_mode = C_MODES[c_mode]
    o.s_dtype = S_DTYPES[s_dtype]
    o.s_per_level = int(bool(s_per_level))
    o.block_threads = int(block_threads)
    o.cluster_size = int(cluster_size)
    o.grid_clusters = int(grid_clusters)
    o.elems_per_thread = int(elems_per_thread)
    o.profile = int(bool(profile))
    o.col_sums = COL_SUMS[col_sums]
    o.schedule = SCHEDULES[schedule]
    o.kappa = float(kappa)
    o.wait_limit_ns = int(wait_limit_ns)
    o.ctas_per_sm = int(ctas_per_sm)
    o.debug_bounds = int(bool(debug_bounds))
    return o


def workspace_bytes(N: int, L: int, **opt) -> int:
    o = options(**opt)
    out = ctypes.c_size_t(0)
    check(lib.hap_workspace_bytes(N, L, ctypes.byref(o), ctypes.byref(out)), "hap_workspace_bytes")
    return out.value


class HAP:
    """One HAP problem: N points, L levels, damping lambda (Algorithm 1 inputs).

    prefs: L preferences (one per level) or an (L, N) array of per-point ones.
    The workspace is a torch uint8 tensor on ``device``; work runs on the
    torch stream current at construction (or ``stream``)."""

    def __init__(self, N: int, L: int, prefs=None, damping: float = 0.5, device="cuda",
                 stream: torch.cuda.Stream | None = None, **opt):
        self.N, self.L, self.damping = int(N), int(L), float(damping)
        self.device = torch.device(device)
        self._opt = options(**opt)
        self.opt = dict(opt)
        with torch.cuda.device(self.device):
            out = ctypes.c_size_t(0)
            check(lib.hap_workspace_bytes(self.N, self.L, ctypes.byref(self._opt), ctypes.byref(out)),
                  "hap_workspace_bytes")
            self.workspace = torch.empty(out.value, dtype=torch.uint8, device=self.device)
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            # construction synchronises its own stream, so wait for the workspace allocation
            self.stream.synchronize()
            h = ctypes.c_void_p()
            check(lib.hap_create(self.N, self.L, None, self.damping, ctypes.byref(self._opt),
                                 _ptr(self.workspace), out.value, ctypes.byref(h)), "hap_create")
            self._h = h
            check(lib.hap_set_stream(self._h, ctypes.c_void_p(self.stream.cuda_stream)), "hap_set_stream")
        if prefs is not None:
            self.set_preferences(prefs)

    # -- lifetime -----------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib.hap_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- inputs -------------------------------------------------------------
    def set_preferences(self, prefs):
        import numpy as np
        p = np.ascontiguousarray(np.asarray(prefs, dtype=np.float32))
        if p.shape == (self.L,):
            per_point = 0
        elif p.shape == (self.L, self.N):
            per_point = 1
        else:
            raise ValueError(f"prefs must have shape ({self.L},) or ({self.L}, {self.N})")
        check(lib.hap_set_preferences(self._h, p.ctypes.data_as(ctypes.c_void_p), per_point), "hap_set_preferences")

    def set_cluster_preferences(self, c0):
        import numpy as np
        c = np.ascontiguousarray(np.asarray(c0, dtype=np.float32).reshape(self.L, self.N))
        check(lib.hap_set_cluster_preferences(self._h, c.ctypes.data_as(ctypes.c_void_p)), "hap_set_cluster_preferences")

    def set_similarity(self, S: torch.Tensor, level: int = -1):
        if S.device != self.device or S.dim() != 2 or S.shape[0] != self.N or S.stride(1) != 1:
            raise ValueError("S must be an (N, >=N) row-major tensor on the context's device")
        dt = {torch.float32: 0, torch.bfloat16: 1}[S.dtype]
        check(lib.hap_set_similarity(self._h, int(level), _ptr(S), S.stride(0), dt), "hap_set_similarity")

    def build_similarity(self, X: torch.Tensor, mode: str = "bf16_split"):
        """X: (N, d) float32 on the context's device, or on the host (the
        library copies it in on its stream)."""
        if X.device not in (self.device, torch.device("cpu")) or X.dtype != torch.float32 or X.dim() != 2 or \
                X.shape[0] != self.N:
            raise ValueError("X must be an (N, d) float32 tensor on the context's device or on the host")
        X = X.contiguous()
        check(lib.hap_build_similarity(self._h, _ptr(X), X.shape[1], SBUILD[mode]), "hap_build_similarity")

    def get_similarity(self, level: int = 0) -> torch.Tensor:
        """The (N, N) float32 similarity the iterations use at ``level``."""
        out = torch.empty((self.N, self.N), dtype=torch.float32, device=self.device)
        check(lib.hap_get_similarity(self._h, int(level), _ptr(out)), "hap_get_similarity")
        self.sync()
        return out

    # -- iteration and outputs -------------------------------------------------
    def iterate(self, n: int = 1):
        check(lib.hap_iterate(self._h, int(n)), "hap_iterate")

    def exemplars(self, out: torch.Tensor | None = None) -> torch.Tensor:
        """Eq. 2.8 assignments, int32 (L, N).  A CPU ``out`` (ideally pinned)
        receives them by a device-to-host copy and the call synchronises."""
        if out is None:
            out = torch.empty((self.L, self.N), dtype=torch.int32, device=self.device)
        if out.dtype != torch.int32 or tuple(out.shape) != (self.L, self.N) or not out.is_contiguous():
            raise ValueError("out must be a contiguous int32 (L, N) tensor")
        check(lib.hap_exemplars(self._h, _ptr(out), 1 if out.device.type == "cpu" else 0), "hap_exemplars")
        return out

    def net_similarity(self):
        import numpy as np
        ns = np.zeros(self.L, dtype=np.float64)
        check(lib.hap_net_similarity(self._h, ns.ctypes.data_as(ctypes.c_void_p)), "hap_net_similarity")
        return ns

    def acceptance(self):
        """(self-consistent points, exemplars) per level of the current assignment."""
        import numpy as np
        cons = np.zeros(self.L, dtype=np.int64)
        ex = np.zeros(self.L, dtype=np.int64)
        check(lib.hap_acceptance(self._h, cons.ctypes.data_as(ctypes.c_void_p), ex.ctypes.data_as(ctypes.c_void_p)),
              "hap_acceptance")
        return cons, ex

    def get_state(self):
        A = torch.empty((self.L, self.N, self.N), dtype=torch.float32, device=self.device)
        R = torch.empty_like(A)
        vecs = torch.empty((3, self.L, self.N), dtype=torch.float32, device=self.device)
        it = ctypes.c_int64(0)
        check(lib.hap_get_state(self._h, _ptr(A), _ptr(R), _ptr(vecs), ctypes.byref(it)), "hap_get_state")
        self.sync()
        return {"A": A, "R": R, "c": vecs[0], "tau": vecs[1], "phi": vecs[2], "t": it.value}

    def set_state(self, A, R, c, t: int, tau=None, phi=None):
        vecs = torch.zeros((3, self.L, self.N), dtype=torch.float32, device=self.device)
        vecs[0] = torch.as_tensor(c, dtype=torch.float32, device=self.device)
        if tau is not None:
            vecs[1] = torch.as_tensor(tau, dtype=torch.float32, device=self.device)
        if phi is not None:
            vecs[2] = torch.as_tensor(phi, dtype=torch.float32, device=self.device)
        A = torch.as_tensor(A, dtype=torch.float32, device=self.device).contiguous()
        R = torch.as_tensor(R, dtype=torch.float32, device=self.device).contiguous()
        self.stream.synchronize()
        check(lib.hap_set_state(self._h, _ptr(A), _ptr(R), _ptr(vecs), int(t)), "hap_set_state")
        self.sync()

    def set_wait_limit(self, ns: int):
        """Limit of the row pass's bounded device waits, in ns (0 = 2 s)."""
        check(lib.hap_set_wait_limit(self._h, int(ns)), "hap_set_wait_limit")

    def sync(self):
        check(lib.hap_sync(self._h), "hap_sync")

    def query(self, key: int) -> int:
        v = ctypes.c_int64(0)
        check(lib.hap_query(self._h, key, ctypes.byref(v)), "hap_query")
        return v.value

    @property
    def shape(self):
        return {"block_threads": self.query(Q_BLOCK_THREADS), "cluster_size": self.query(Q_CLUSTER_SIZE),
                "grid_clusters": self.query(Q_GRID_CLUSTERS), "ld": self.query(Q_LD),
                "elems_per_thread": self.query(Q_ELEMS_PER_THREAD),
                "col_sums": {1: "smem", 2: "tmem"}[self.query(Q_COL_SUMS)], "stages": self.query(Q_STAGES),
                "ctas_per_sm": self.query(Q_CTAS_PER_SM)}

    @property
    def launches(self) -> int:
        """Kernels this context has launched so far."""
        return self.query(Q_LAUNCHES)

    @property
    def iterations(self) -> int:
        return self.query(Q_ITER)

    def row_pass_time(self, reset: bool = True):
        ms = ctypes.c_double(0.0)
        n = ctypes.c_int64(0)
        check(lib.hap_row_pass_time(self._h, ctypes.byref(ms), ctypes.byref(n), int(reset)), "hap_row_pass_time")
        return ms.value, n.value


def iterate_noalloc(N: int, L: int, damping: float, c_mode: str, S: torch.Tensor, pref: torch.Tensor,
                    A: torch.Tensor, R: torch.Tensor, c: torch.Tensor, tau: torch.Tensor, phi: torch.Tensor,
                    t0: int, n: int, stream: torch.cuda.Stream | None = None) -> None:
    """hap_iterate_noalloc on caller-owned tensors (padded layout, ld = N
    rounded up to 32): S (N, ld) float32/bfloat16, pref/c/tau/phi (L, ld),
    A/R (L, N, ld) float32.  Runs n iterations after t0, allocating nothing."""
    ld = (N + 31) // 32 * 32
    if S.device.type != "cuda" or S.dtype not in (torch.float32, torch.bfloat16):
        raise ValueError("S must be a float32 or bfloat16 CUDA tensor")
    for name, t, shape in (("S", S, (N, ld)), ("pref", pref, (L, ld)), ("A", A, (L, N, ld)), ("R", R, (L, N, ld)),
                           ("c", c, (L, ld)), ("tau", tau, (L, ld)), ("phi", phi, (L, ld))):
        if tuple(t.shape) != shape or not t.is_contiguous() or t.device != S.device:
            raise ValueError(f"{name} must be a contiguous tensor of shape {shape} on {S.device}")
        if name != "S" and t.dtype != torch.float32:
            raise ValueError(f"{name} must be float32")
    dt = {torch.float32: 0, torch.bfloat16: 1}[S.dtype]
    with torch.cuda.device(S.device):  # the library uses the scratch array of the current device
        st = stream if stream is not None else torch.cuda.current_stream(S.device)
        check(lib.hap_iterate_noalloc(int(N), int(L), float(damping), C_MODES[c_mode], _ptr(S), dt, _ptr(pref),
                                      _ptr(A), _ptr(R), _ptr(c), _ptr(tau), _ptr(phi), int(t0), int(n),
                                      ctypes.c_void_p(st.cuda_stream)), "hap_iterate_noalloc")


class HAPBatch:
    """Many independent HAP problems (N[b] points, L[b] levels) advanced by one
    persistent launch per iteration (hap_batch_* in the C ABI)."""

    def __init__(self, N, L, damping: float = 0.5, device="cuda", stream: torch.cuda.Stream | None = None,
                 c_mode="paper", s_dtype="f32", **opt):
        import numpy as np
        self.N = [int(x) for x in N]
        self.L = [int(x) for x in L]
        self.B = len(self.N)
        self.device = torch.device(device)
        o = options(c_mode=c_mode, s_dtype=s_dtype, **opt)
        n_arr = np.ascontiguousarray(self.N, dtype=np.int64)
        l_arr = np.ascontiguousarray(self.L, dtype=np.int32)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            h = ctypes.c_void_p()
            check(lib.hap_batch_create(self.B, n_arr.ctypes.data_as(ctypes.c_void_p), l_arr.ctypes.data_as(ctypes.c_void_p),
                                       float(damping), ctypes.byref(o), ctypes.byref(h)), "hap_batch_create")
            self._h = h
            check(lib.hap_batch_set_stream(self._h, ctypes.c_void_p(self.stream.cuda_stream)), "hap_batch_set_stream")

    def close(self):
        if getattr(self, "_h", None):
            lib.hap_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_preferences(self, prefs):
        """One preference per (instance, level), instance-major."""
        import numpy as np
        p = np.ascontiguousarray(np.concatenate([np.broadcast_to(np.asarray(x, dtype=np.float32), (l,))
                                                 for x, l in zip(prefs, self.L)]))
        check(lib.hap_batch_set_preferences(self._h, p.ctypes.data_as(ctypes.c_void_p)), "hap_batch_set_preferences")

    def set_similarity(self, b: int, S: torch.Tensor):
        dt = {torch.float32: 0, torch.bfloat16: 1}[S.dtype]
        check(lib.hap_batch_set_similarity(self._h, int(b), _ptr(S), S.stride(0), dt), "hap_batch_set_similarity")

    def build_similarity(self, X: torch.Tensor, mode: str = "bf16_split"):
        """X: (sum N, d) float32 CUDA tensor, instance-major rows."""
        X = X.contiguous()
        check(lib.hap_batch_build_similarity(self._h, _ptr(X), X.shape[1], SBUILD[mode]), "hap_batch_build_similarity")

    def iterate(self, n: int = 1):
        check(lib.hap_batch_iterate(self._h, int(n)), "hap_batch_iterate")

    def tune(self) -> float:
        ms = ctypes.c_double(0.0)
        check(lib.hap_batch_tune(self._h, ctypes.byref(ms)), "hap_batch_tune")
        return ms.value

    def set_wait_limit(self, ns: int):
        """Limit of the batched row pass's bounded device waits, in ns (0 = 2 s)."""
        check(lib.hap_batch_set_wait_limit(self._h, int(ns)), "hap_batch_set_wait_limit")

    def set_tile(self, elems_per_thread: int):
        """Columns per thread of the row pass (16 or 8); resets the messages."""
        check(lib.hap_batch_set_tile(self._h, int(elems_per_thread)), "hap_batch_set_tile")

    @property
    def tile(self) -> dict:
        return {"elems_per_thread": self.query(Q_ELEMS_PER_THREAD), "items_per_cta": self.query(Q_BATCH_ITEMS_PER_CTA)}

    def exemplars(self, out: torch.Tensor | None = None):
        """List of int32 (L[b], N[b]) tensors (views of one flat buffer)."""
        total = sum(n * l for n, l in zip(self.N, self.L))
        if out is None:
            out = torch.empty(total, dtype=torch.int32, device=self.device)
        check(lib.hap_batch_exemplars(self._h, _ptr(out), 1 if out.device.type == "cpu" else 0), "hap_batch_exemplars")
        res, q = [], 0
        for n, l in zip(self.N, self.L):
            res.append(out[q:q + n * l].view(l, n))
            q += n * l
        return res

    def net_similarity(self):
        import numpy as np
        ns = np.zeros(sum(self.L), dtype=np.float64)
        check(lib.hap_batch_net_similarity(self._h, ns.ctypes.data_as(ctypes.c_void_p)), "hap_batch_net_similarity")
        out, q = [], 0
        for l in self.L:
            out.append(ns[q:q + l])
            q += l
        return out

    def get_state(self, b: int):
        n, l = self.N[b], self.L[b]
        A = torch.empty((l, n, n), dtype=torch.float32, device=self.device)
        R = torch.empty_like(A)
        vecs = torch.empty((3, l, n), dtype=torch.float32, device=self.device)
        it = ctypes.c_int64(0)
        check(lib.hap_batch_get_state(self._h, int(b), _ptr(A), _ptr(R), _ptr(vecs), ctypes.byref(it)),
              "hap_batch_get_state")
        check(lib.hap_batch_sync(self._h), "hap_batch_sync")
        return {"A": A, "R": R, "c": vecs[0], "tau": vecs[1], "phi": vecs[2], "t": it.value}

    def query(self, key: int) -> int:
        v = ctypes.c_int64(0)
        check(lib.hap_batch_query(self._h, key, ctypes.byref(v)), "hap_batch_query")
        return v.value

    def sync(self):
        check(lib.hap_batch_sync(self._h), "hap_batch_sync")


# ---- learned candidate proposal and sparse HAP -------------------------------
def _stream_ptr(device, stream=None):
    st = stream if stream is not None else torch.cuda.current_stream(device)
    return ctypes.c_void_p(st.cuda_stream)


KNN_METHODS = {"auto": 0, "cuda_cores": 1, "tensor_cores": 2}


def proposal_launches() -> int:
    """Kernels launched so far through the stateless proposal functions."""
    return int(lib.hap_proposal_launches())


def knn(X: torch.Tensor, M: int, stream=None, method: str = "auto"):
    """Exact M nearest neighbours (squared Euclidean, self excluded):
    (idx int32 (N, M), dist float32 (N, M)) on X's device."""
    X = X.contiguous()
    N, d = X.shape
    idx = torch.empty((N, M), dtype=torch.int32, device=X.device)
    dist = torch.empty((N, M), dtype=torch.float32, device=X.device)
    check(lib.hap_knn_with(_ptr(X), N, d, int(M), KNN_METHODS[method], _ptr(idx), _ptr(dist),
                           _stream_ptr(X.device, stream)), "hap_knn_with")
    return idx, dist


def knn_subset(X: torch.Tensor, subset: torch.Tensor, M: int, stream=None, method: str = "auto"):
    """For every point, its M nearest members of `subset` (global indices)."""
    X = X.contiguous()
    N, d = X.shape
    idx = torch.empty((N, M), dtype=torch.int32, device=X.device)
    dist = torch.empty((N, M), dtype=torch.float32, device=X.device)
    check(lib.hap_knn_subset_with(_ptr(X), N, d, _ptr(subset.contiguous()), subset.numel(), int(M),
                                  KNN_METHODS[method], _ptr(idx), _ptr(dist), _stream_ptr(X.device, stream)),
          "hap_knn_subset_with")
    return idx, dist


def top_scores(score: torch.Tensor, H: int, stream=None):
    hubs = torch.empty(int(H), dtype=torch.int32, device=score.device)
    check(lib.hap_top_scores(_ptr(score.contiguous()), score.numel(), int(H), _ptr(hubs),
                             _stream_ptr(score.device, stream)), "hap_top_scores")
    return hubs


def select_hub_candidates(pool: torch.Tensor, hubnn: torch.Tensor, K: int, K_near: int, stream=None):
    N, Mp = pool.shape
    cand = torch.empty((N, K), dtype=torch.int32, device=pool.device)
    check(lib.hap_select_hub_candidates(_ptr(pool.contiguous()), N, Mp, _ptr(hubnn.contiguous()), hubnn.shape[1], int(K),
                                        int(K_near), _ptr(cand), _stream_ptr(pool.device, stream)),
          "hap_select_hub_candidates")
    return cand


def exemplar_points(e: torch.Tensor, N: int, stream=None):
    """The distinct points among the exemplar indices e (any shape, device
    int32), in increasing order: a device int32 tensor (a view of length
    count)."""
    e = e.contiguous()
    points = torch.empty(int(N), dtype=torch.int32, device=e.device)
    count = ctypes.c_int64()
    check(lib.hap_exemplar_points(_ptr(e), e.numel(), int(N), _ptr(points), ctypes.byref(count),
                                  _stream_ptr(e.device, stream)), "hap_exemplar_points")
    return points[: count.value]


def refine_candidates(X: torch.Tensor, pool: torch.Tensor, e: torch.Tensor, K: int, K_near: int, stream=None):
    """Candidates for a second sparse solve: every row keeps itself, its
    K_near nearest neighbours (pool) and its nearest exemplars of the first
    solve (e, all levels) as hubs (up to K in all)."""
    hubs = exemplar_points(e, X.shape[0], stream)
    hubnn, _ = knn_subset(X, hubs, min(int(K), hubs.numel()), stream)
    return select_hub_candidates(pool, hubnn, K, K_near, stream)


def knn_features(dist: torch.Tensor, F: int, stream=None):
    """(feats (N, F), log_scale) with feats = log(dist[:, :F]) - mean log(dist[:, F-1])."""
    N, M = dist.shape
    feats = torch.empty((N, F), dtype=torch.float32, device=dist.device)
    ls = ctypes.c_float(0.0)
    check(lib.hap_knn_features(_ptr(dist.contiguous()), N, M, int(F), _ptr(feats), ctypes.byref(ls),
                               _stream_ptr(dist.device, stream)), "hap_knn_features")
    return feats, ls.value


def mlp_init_params(F: int, seed: int = 0, width: int = 128):
    """Flat FP32 initial parameters: uniform(+-1/sqrt(fan_in)) weights, zero biases."""
    import numpy as np
    rng = np.random.default_rng(seed)
    a1, a2 = 1.0 / np.sqrt(F), 1.0 / np.sqrt(width)
    parts = [rng.uniform(-a1, a1, F * width), np.zeros(width), rng.uniform(-a2, a2, width * width),
             np.zeros(width), rng.uniform(-a2, a2, width), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


class MLP:
    """The proposal network (hap_mlp_*): width 128, BF16 weights, FP32 accumulation."""

    def __init__(self, F: int, theta0=None, seed: int = 0, device="cuda", stream=None):
        import numpy as np
        self.F = int(F)
        self.device = torch.device(device)
        th = mlp_init_params(F, seed) if theta0 is None else np.ascontiguousarray(np.asarray(theta0, dtype=np.float32))
        with torch.cuda.device(self.device):
            h = ctypes.c_void_p()
            check(lib.hap_mlp_create(self.F, th.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)), "hap_mlp_create")
            self._h = h
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            check(lib.hap_mlp_set_stream(self._h, ctypes.c_void_p(self.stream.cuda_stream)), "hap_mlp_set_stream")
        P = ctypes.c_int64(0)
        check(lib.hap_mlp_num_params(self._h, ctypes.byref(P)), "hap_mlp_num_params")
        self.P = P.value

    def close(self):
        if getattr(self, "_h", None):
            lib.hap_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        import numpy as np
        th = np.empty(self.P, dtype=np.float32)
        check(lib.hap_mlp_get_params(self._h, th.ctypes.data_as(ctypes.c_void_p)), "hap_mlp_get_params")
        return th

    def forward(self, feats: torch.Tensor) -> torch.Tensor:
        feats = feats.contiguous()
        out = torch.empty(feats.shape[0], dtype=torch.float32, device=self.device)
        check(lib.hap_mlp_forward(self._h, _ptr(feats), feats.shape[0], _ptr(out)), "hap_mlp_forward")
        return out

    def gradients(self, feats: torch.Tensor, labels: torch.Tensor, pos_weight: float):
        import numpy as np
        g = np.empty(self.P, dtype=np.float32)
        loss = ctypes.c_float(0.0)
        check(lib.hap_mlp_gradients(self._h, _ptr(feats.contiguous()), _ptr(labels.contiguous()), feats.shape[0],
                                    float(pos_weight), g.ctypes.data_as(ctypes.c_void_p), ctypes.byref(loss)),
              "hap_mlp_gradients")
        return g, loss.value

    def train_step(self, feats: torch.Tensor, labels: torch.Tensor, pos_weight: float, lr: float, want_loss=False):
        loss = ctypes.c_float(0.0)
        check(lib.hap_mlp_train_step(self._h, _ptr(feats), _ptr(labels), feats.shape[0], float(pos_weight), float(lr),
                                     ctypes.byref(loss) if want_loss else None), "hap_mlp_train_step")
        return loss.value if want_loss else None


def select_candidates(pool: torch.Tensor, K: int, K_near: int, score: torch.Tensor | None = None, stream=None):
    N, M = pool.shape
    cand = torch.empty((N, K), dtype=torch.int32, device=pool.device)
    check(lib.hap_select_candidates(_ptr(pool.contiguous()), N, M, _ptr(score) if score is not None else None, int(K),
                                    int(K_near), _ptr(cand), _stream_ptr(pool.device, stream)), "hap_select_candidates")
    return cand


def net_similarity_points(X: torch.Tensor, e: torch.Tensor, pref: torch.Tensor, stream=None):
    """FP64 NS per level of assignment e (L, N) from the points X (N, d), pref (L, N)."""
    import numpy as np
    L, N = e.shape
    ns = np.zeros(L, dtype=np.float64)
    check(lib.hap_net_similarity_points(_ptr(X.contiguous()), N, X.shape[1], L, _ptr(e.contiguous()),
                                        _ptr(pref.contiguous()), ns.ctypes.data_as(ctypes.c_void_p),
                                        _stream_ptr(X.device, stream)), "hap_net_similarity_points")
    return ns


class HAPSparse:
    """Sparse HAP over a K-candidate graph (hap_sparse_*)."""

    def __init__(self, N: int, L: int, K: int, prefs=None, damping: float = 0.5, c_mode="paper", device="cuda",
                 stream=None):
        import numpy as np
        self.N, self.L, self.K = int(N), int(L), int(K)
        self.device = torch.device(device)
        with torch.cuda.device(self.device):
            h = ctypes.c_void_p()
            check(lib.hap_sparse_create(self.N, self.L, self.K, None, float(damping), C_MODES[c_mode], ctypes.byref(h)),
                  "hap_sparse_create")
            self._h = h
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            check(lib.hap_sparse_set_stream(self._h, ctypes.c_void_p(self.stream.cuda_stream)), "hap_sparse_set_stream")
        if prefs is not None:
            self.set_preferences(prefs)

    def close(self):
        if getattr(self, "_h", None):
            lib.hap_sparse_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_profile(self, on: bool = True):
        """Time every later iteration's four steps with CUDA events."""
        check(lib.hap_sparse_set_profile(self._h, int(bool(on))), "hap_sparse_set_profile")

    def profile_times(self, reset: bool = True):
        """({"row_pass": ms, "column_statistics": ms}, iterations) summed over
        the profiled iterations."""
        import numpy as np
        ms = np.zeros(2, dtype=np.float64)
        n = ctypes.c_int64(0)
        check(lib.hap_sparse_profile_times(self._h, ms.ctypes.data_as(ctypes.c_void_p), ctypes.byref(n), int(reset)),
              "hap_sparse_profile_times")
        return dict(zip(("row_pass", "column_statistics"), ms.tolist())), n.value

    def set_preferences(self, prefs):
        import numpy as np
        p = np.ascontiguousarray(np.asarray(prefs, dtype=np.float32))
        per_point = 1 if p.ndim == 2 else 0
        check(lib.hap_sparse_set_preferences(self._h, p.ctypes.data_as(ctypes.c_void_p), per_point),
              "hap_sparse_set_preferences")

    def set_candidates(self, cand: torch.Tensor, X: torch.Tensor):
        self._X = X.contiguous()
        check(lib.hap_sparse_set_candidates(self._h, _ptr(cand.contiguous()), _ptr(self._X), self._X.shape[1]),
              "hap_sparse_set_candidates")

    def iterate(self, n: int = 1):
        check(lib.hap_sparse_iterate(self._h, int(n)), "hap_sparse_iterate")

    def exemplars(self, out: torch.Tensor | None = None):
        if out is None:
            out = torch.empty((self.L, self.N), dtype=torch.int32, device=self.device)
        check(lib.hap_sparse_exemplars(self._h, _ptr(out), 1 if out.device.type == "cpu" else 0), "hap_sparse_exemplars")
        return out

    def net_similarity(self):
        import numpy as np
        ns = np.zeros(self.L, dtype=np.float64)
        check(lib.hap_sparse_net_similarity(self._h, ns.ctypes.data_as(ctypes.c_void_p)), "hap_sparse_net_similarity")
        return ns

    @property
    def launches(self) -> int:
        v = ctypes.c_int64(0)
        check(lib.hap_sparse_query(self._h, Q_LAUNCHES, ctypes.byref(v)), "hap_sparse_query")
        return v.value

    def get_state(self):
        A = torch.empty((self.L, self.N, self.K), dtype=torch.float32, device=self.device)
        R = torch.empty_like(A)
        vecs = torch.empty((3, self.L, self.N), dtype=torch.float32, device=self.device)
        it = ctypes.c_int64(0)
        check(lib.hap_sparse_get_state(self._h, _ptr(A), _ptr(R), _ptr(vecs), ctypes.byref(it)), "hap_sparse_get_state")
        self.stream.synchronize()
        return {"A": A, "R": R, "c": vecs[0], "tau": vecs[1], "phi": vecs[2], "t": it.value}


class HAPBand:
    """Rows row0 .. row0 + nrows - 1 of an N-point HAP problem (the row
    partition of §3).  One iteration is ``rows(xch)`` on every band, then
    ``columns(xch_all, bounds)`` on every band with all bands' exchange
    buffers in band order: an all-gather of ``xch`` between devices, or, for
    bands on one device, each band writing straight into its slot of one
    ``(P, 4, L, ld)`` tensor (``BandGroup``)."""

    def __init__(self, N: int, row0: int, nrows: int, L: int, prefs=None, damping: float = 0.5, device="cuda",
                 stream: torch.cuda.Stream | None = None, **opt):
        import numpy as np
        self.N, self.row0, self.nrows, self.L = int(N), int(row0), int(nrows), int(L)
        self.damping = float(damping)
        self.device = torch.device(device)
        self._opt = options(**opt)
        p = None if prefs is None else np.ascontiguousarray(np.asarray(prefs, dtype=np.float32).reshape(self.L))
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            h = ctypes.c_void_p()
            check(lib.hap_band_create(self.N, self.row0, self.nrows, self.L,
                                      None if p is None else p.ctypes.data_as(ctypes.c_void_p), self.damping,
                                      ctypes.byref(self._opt), ctypes.byref(h)), "hap_band_create")
            self._h = h
            check(lib.hap_band_set_stream(self._h, ctypes.c_void_p(self.stream.cuda_stream)), "hap_band_set_stream")
        n = ctypes.c_int64(0)
        check(lib.hap_band_exchange_floats(self._h, ctypes.byref(n)), "hap_band_exchange_floats")
        self.exchange_floats = n.value
        self.ld = self.query(Q_LD)

    def close(self):
        if getattr(self, "_h", None):
            lib.hap_band_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_similarity(self, S_rows: torch.Tensor):
        """S_rows: (nrows, >=N) row-major rows row0.. of the problem's S."""
        if S_rows.device != self.device or S_rows.dim() != 2 or S_rows.shape[0] != self.nrows or \
                S_rows.shape[1] < self.N or S_rows.stride(1) != 1:
            raise ValueError("S_rows must be an (nrows, >=N) row-major tensor on the band's device")
        dt = {torch.float32: 0, torch.bfloat16: 1}[S_rows.dtype]
        self.stream.synchronize()
        check(lib.hap_band_set_similarity(self._h, _ptr(S_rows), S_rows.stride(0), dt), "hap_band_set_similarity")

    def rows(self, xch: torch.Tensor):
        """Row pass of one iteration; writes the band's exchange buffer into
        ``xch`` (float32, exchange_floats elements, on the band's device)."""
        if xch.device != self.device or xch.dtype != torch.float32 or not xch.is_contiguous() or \
                xch.numel() != self.exchange_floats:
            raise ValueError("xch must be a contiguous float32 tensor of exchange_floats elements")
        check(lib.hap_band_rows(self._h, _ptr(xch)), "hap_band_rows")

    def columns(self, xch_all: torch.Tensor, bounds):
        """Column statistics from every band's buffer (P, exchange_floats) in
        band order; bounds: the P + 1 row boundaries of the bands."""
        import numpy as np
        b = np.ascontiguousarray(np.asarray(bounds, dtype=np.int64))
        P = len(b) - 1
        if xch_all.device != self.device or xch_all.dtype != torch.float32 or not xch_all.is_contiguous() or \
                xch_all.numel() != P * self.exchange_floats:
            raise ValueError("xch_all must be a contiguous float32 (P, exchange_floats) tensor")
        check(lib.hap_band_columns(self._h, _ptr(xch_all), P, b.ctypes.data_as(ctypes.c_void_p)), "hap_band_columns")

    def get_state(self):
        A = torch.empty((self.L, self.nrows, self.N), dtype=torch.float32, device=self.device)
        R = torch.empty_like(A)
        vecs = torch.empty((3, self.L, self.N), dtype=torch.float32, device=self.device)
        it = ctypes.c_int64(0)
        check(lib.hap_band_get_state(self._h, _ptr(A), _ptr(R), _ptr(vecs), ctypes.byref(it)), "hap_band_get_state")
        self.sync()
        return {"A": A, "R": R, "c": vecs[0], "tau": vecs[1], "phi": vecs[2], "t": it.value}

    def exemplars(self) -> torch.Tensor:
        out = torch.empty((self.L, self.nrows), dtype=torch.int32, device=self.device)
        check(lib.hap_band_exemplars(self._h, _ptr(out), 0), "hap_band_exemplars")
        return out

    def sync(self):
        check(lib.hap_band_sync(self._h), "hap_band_sync")

    def query(self, key: int) -> int:
        v = ctypes.c_int64(0)
        check(lib.hap_band_query(self._h, key, ctypes.byref(v)), "hap_band_query")
        return v.value

    @property
    def launches(self) -> int:
        return self.query(Q_LAUNCHES)


class BandGroup:
    """P row bands of one problem on one device, stepped together: every
    band's row pass writes its exchange buffer straight into its slot of one
    (P, 4, L, ld) tensor, which then feeds every band's column statistics."""

    def __init__(self, N: int, L: int, bounds, prefs=None, damping: float = 0.5, device="cuda", **opt):
        self.bounds = [int(x) for x in bounds]
        self.N, self.L = int(N), int(L)
        self.bands = [HAPBand(N, self.bounds[r], self.bounds[r + 1] - self.bounds[r], L, prefs, damping, device,
                              **opt) for r in range(len(self.bounds) - 1)]
        self.xch = torch.empty((len(self.bands), self.bands[0].exchange_floats), dtype=torch.float32,
                               device=self.bands[0].device)

    def set_similarity(self, S: torch.Tensor):
        for r, b in enumerate(self.bands):
            b.set_similarity(S[self.bounds[r]:self.bounds[r + 1]])

    def iterate(self, n: int = 1):
        for _ in range(int(n)):
            for r, b in enumerate(self.bands):
                b.rows(self.xch[r])
            for b in self.bands:
                b.columns(self.xch, self.bounds)

    def get_state(self):
        st = [b.get_state() for b in self.bands]
        own = torch.cat([s["tau"][:, self.bounds[r]:self.bounds[r + 1]] for r, s in enumerate(st)], dim=1)
        return {"A": torch.cat([s["A"] for s in st], dim=1), "R": torch.cat([s["R"] for s in st], dim=1),
                "c": st[0]["c"], "tau": own, "phi": st[0]["phi"], "t": st[0]["t"], "per_band": st}

    def exemplars(self) -> torch.Tensor:
        return torch.cat([b.exemplars() for b in self.bands], dim=1)

    def close(self):
        for b in self.bands:
            b.close()
