"""Thin ctypes binding of ``libkpynq.so`` (declared in ``include/kpynq.h``).

The functions below carry the C names and only marshal arguments: every step
of the K-means iteration runs in the library's CUDA kernels.  Arrays may be
PyTorch tensors (host or CUDA), NumPy arrays, or raw integer addresses; the
library itself tells host from device memory.  If the library has not been
built, loading fails loudly -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libkpynq.so")

KM_OK, KM_EINVAL, KM_ENOMEM, KM_ECUDA, KM_ETIMEOUT, KM_ESTATE = 0, -1, -2, -3, -4, -5
KM_ALGO_FILTERED, KM_ALGO_LLOYD = 0, 1
KM_DTYPE_F32, KM_DTYPE_BF16 = 0, 1
KM_GROUP_CONTIGUOUS, KM_GROUP_CLUSTERED = 0, 1
KM_DENSE_AUTO, KM_DENSE_FP32 = 0, 1
KM_PATH_FILTERED, KM_PATH_DENSE_FP32, KM_PATH_DENSE_TC = 0, 1, 2
(KM_KERNEL_DENSE, KM_KERNEL_MOVES, KM_KERNEL_FILTER, KM_KERNEL_SURVIVOR, KM_KERNEL_UPDATE, KM_KERNEL_OTHER,
 KM_KERNEL_SETTLE, KM_KERNEL_STATS, KM_KERNEL_PROPOSAL) = range(9)
KERNEL_KIND_NAMES = ["dense_assign", "apply_moves", "filter", "survivor", "update", "other", "settle", "stats",
                     "proposal"]
STATUS_NAMES = {0: "KM_OK", -1: "KM_EINVAL", -2: "KM_ENOMEM", -3: "KM_ECUDA", -4: "KM_ETIMEOUT",
                -5: "KM_ESTATE"}


class KMeansError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class kmeans_options(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int32), ("grouping", ctypes.c_int32), ("validate", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("stream", ctypes.c_void_p), ("dense", ctypes.c_int32),
                ("dense_switch", ctypes.c_float), ("dtype", ctypes.c_int32), ("pad0", ctypes.c_int32),
                ("surv_grab", ctypes.c_int32), ("pad1", ctypes.c_int32), ("reserved", ctypes.c_int64 * 3)]


class kmeans_problem(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("N", ctypes.c_int64), ("D", ctypes.c_int32), ("K", ctypes.c_int32),
                ("G", ctypes.c_int32), ("init_centroids", ctypes.c_void_p)]


class kmeans_iter_stats(ctypes.Structure):
    _fields_ = [("iter", ctypes.c_int32), ("done", ctypes.c_int32), ("path", ctypes.c_int32),
                ("n_settle", ctypes.c_int32), ("n_changed", ctypes.c_int64),
                ("n_survivors", ctypes.c_int64), ("n_scanned", ctypes.c_int64), ("n_dist", ctypes.c_int64),
                ("n_recheck", ctypes.c_int64), ("objective", ctypes.c_double), ("max_drift", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def lib():
    """Load libkpynq.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                              "or python -m paper_1905_09345_gb300.build")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.kmeans_default_options.argtypes = [ctypes.POINTER(kmeans_options)]
        L.kmeans_default_options.restype = None
        L.kmeans_selftest_sqrt.argtypes = [ctypes.POINTER(i64)]
        L.kmeans_set_proposal.argtypes = [vp, vp, vp, vp, vp, vp, vp, i32]
        L.kmeans_set_proposal.restype = ctypes.c_int
        L.kmeans_mlp_predict.argtypes = [vp, i64, i32, vp, vp, vp, vp, vp, vp, i32, i32, vp, vp]
        L.kmeans_mlp_predict.restype = ctypes.c_int
        L.kmeans_selftest_sqrt.restype = ctypes.c_int
        L.kmeans_init.argtypes = [ctypes.POINTER(vp), vp, i64, i32, i32, i32, vp, ctypes.POINTER(kmeans_options)]
        L.kmeans_init.restype = ctypes.c_int
        L.kmeans_iterate.argtypes = [vp, ctypes.POINTER(kmeans_iter_stats)]
        L.kmeans_iterate.restype = ctypes.c_int
        L.kmeans_fit.argtypes = [vp, i32, dbl, vp, vp, vp, vp]
        L.kmeans_fit.restype = ctypes.c_int
        L.kmeans_get_labels.argtypes = [vp, vp]
        L.kmeans_get_labels.restype = ctypes.c_int
        L.kmeans_get_centroids.argtypes = [vp, vp]
        L.kmeans_get_centroids.restype = ctypes.c_int
        L.kmeans_get_stats.argtypes = [vp, i32, ctypes.POINTER(kmeans_iter_stats)]
        L.kmeans_get_stats.restype = ctypes.c_int
        L.kmeans_get_bounds.argtypes = [vp, vp, vp, vp]
        L.kmeans_get_bounds.restype = ctypes.c_int
        L.kmeans_get_groups.argtypes = [vp, vp, ctypes.POINTER(i32)]
        L.kmeans_get_groups.restype = ctypes.c_int
        L.kmeans_get_iteration.argtypes = [vp, ctypes.POINTER(i32)]
        L.kmeans_get_iteration.restype = ctypes.c_int
        L.kmeans_get_kernel_count.argtypes = [vp, ctypes.POINTER(i64)]
        L.kmeans_get_kernel_count.restype = ctypes.c_int
        L.kmeans_reset.argtypes = [vp, vp]
        L.kmeans_reset.restype = ctypes.c_int
        L.kmeans_get_profile.argtypes = [vp, i32, ctypes.POINTER(i64), ctypes.POINTER(dbl)]
        L.kmeans_get_profile.restype = ctypes.c_int
        L.kmeans_lloyd_step_noalloc.argtypes = [vp, i64, i32, vp, i32, vp, vp, vp, vp]
        L.kmeans_lloyd_step_noalloc.restype = ctypes.c_int
        L.kmeans_destroy.argtypes = [vp]
        L.kmeans_destroy.restype = None
        L.kmeans_last_error.argtypes = [vp]
        L.kmeans_last_error.restype = ctypes.c_char_p
        L.kmeans_launch_count.argtypes = []
        L.kmeans_launch_count.restype = i64
        L.kmeans_batch_init.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(kmeans_problem),
                                        ctypes.POINTER(kmeans_options), ctypes.c_char_p]
        L.kmeans_batch_init.restype = ctypes.c_int
        L.kmeans_batch_fit.argtypes = [vp, i32, dbl]
        L.kmeans_batch_fit.restype = ctypes.c_int
        L.kmeans_batch_get.argtypes = [vp, i32, vp, vp, vp, vp]
        L.kmeans_batch_get.restype = ctypes.c_int
        L.kmeans_batch_reset.argtypes = [vp]
        L.kmeans_batch_reset.restype = ctypes.c_int
        L.kmeans_batch_get_tuning.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(i32),
                                              ctypes.POINTER(i32)]
        L.kmeans_batch_get_tuning.restype = ctypes.c_int
        L.kmeans_batch_get_switch.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_float)]
        L.kmeans_batch_get_switch.restype = ctypes.c_int
        L.kmeans_batch_destroy.argtypes = [vp]
        L.kmeans_batch_destroy.restype = None
        L.kmeans_batch_last_error.argtypes = [vp]
        L.kmeans_batch_last_error.restype = ctypes.c_char_p
        L.kmeans_shard_assign.argtypes = [vp, dbl, vp, vp, vp, ctypes.POINTER(i64)]
        L.kmeans_shard_assign.restype = ctypes.c_int
        L.kmeans_shard_update.argtypes = [vp, i32, vp, vp, vp, i64, ctypes.POINTER(kmeans_iter_stats),
                                          ctypes.POINTER(dbl)]
        L.kmeans_shard_update.restype = ctypes.c_int
        L.kmeans_init_kmeanspp.argtypes = [vp, i64, i32, i32, vp, vp, vp, vp]
        L.kmeans_init_kmeanspp.restype = ctypes.c_int
        L.kmeans_selftest_timeout.argtypes = [i32]
        L.kmeans_selftest_timeout.restype = ctypes.c_int
        L.kmeans_debug_fail_alloc.argtypes = [i64]
        L.kmeans_debug_fail_alloc.restype = None
        u64, f32 = ctypes.c_uint64, ctypes.c_float
        L.kmeans_mlp_create.argtypes = [ctypes.POINTER(vp), i32, i32, i32, u64, vp]
        L.kmeans_mlp_create.restype = ctypes.c_int
        L.kmeans_mlp_set_params.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.kmeans_mlp_set_params.restype = ctypes.c_int
        L.kmeans_mlp_get_params.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.kmeans_mlp_get_params.restype = ctypes.c_int
        L.kmeans_mlp_gradient.argtypes = [vp, vp, vp, i32, ctypes.POINTER(dbl), vp]
        L.kmeans_mlp_gradient.restype = ctypes.c_int
        L.kmeans_mlp_train.argtypes = [vp, vp, i64, vp, i32, i64, i32, f32, u64, ctypes.POINTER(dbl),
                                       ctypes.POINTER(dbl)]
        L.kmeans_mlp_train.restype = ctypes.c_int
        L.kmeans_mlp_predict_net.argtypes = [vp, vp, i64, vp]
        L.kmeans_mlp_predict_net.restype = ctypes.c_int
        L.kmeans_mlp_destroy.argtypes = [vp]
        L.kmeans_mlp_destroy.restype = None
        L.kmeans_mlp_last_error.argtypes = [vp]
        L.kmeans_mlp_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _addr(a) -> int | None:
    """Address of a tensor / array / integer (None stays None)."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):  # torch.Tensor
        if not a.is_contiguous():
            raise ValueError("arrays must be contiguous")
        return a.data_ptr()
    if hasattr(a, "ctypes"):  # numpy
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"cannot take the address of {type(a)}")


def _check(rc: int, ctx=None):
    if rc != KM_OK:
        msg = lib().kmeans_last_error(ctx).decode(errors="replace")
        raise KMeansError(rc, msg)


# ---------------------------------------------------------------------------
# C-named wrappers
# ---------------------------------------------------------------------------
def kmeans_default_options() -> kmeans_options:
    o = kmeans_options()
    lib().kmeans_default_options(ctypes.byref(o))
    return o


def _dtype_of(X, dtype):
    """KM_DTYPE_* of X: explicit, else bfloat16 for a torch bfloat16 tensor,
    else FP32 (a uint16 numpy array of bfloat16 bit patterns needs
    dtype=KM_DTYPE_BF16)."""
    if dtype is not None:
        return int(dtype)
    return KM_DTYPE_BF16 if str(getattr(X, "dtype", "")) == "torch.bfloat16" else KM_DTYPE_F32



def kmeans_selftest_sqrt() -> int:
    """Failures of the square-root bounds over every non-negative float on the
    current device (0 expected)."""
    v = ctypes.c_int64(-1)
    _check(lib().kmeans_selftest_sqrt(ctypes.byref(v)), None)
    return v.value


MLP_NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


def kmeans_set_proposal(ctx, W1, b1, W2, b2, W3, b3, hidden: int) -> None:
    """Set (or, with all six None, remove) the learned group proposal."""
    _check(lib().kmeans_set_proposal(ctx, _addr(W1), _addr(b1), _addr(W2), _addr(b2), _addr(W3), _addr(b3),
                                     hidden), ctx)


def kmeans_mlp_predict(X, N: int, D: int, W1, b1, W2, b2, W3, b3, hidden: int, classes: int, pred,
                       stream=None) -> None:
    """The proposal MLP's argmax group for every point (device arrays)."""
    st = stream if isinstance(stream, int) or stream is None else stream.cuda_stream
    _check(lib().kmeans_mlp_predict(_addr(X), N, D, _addr(W1), _addr(b1), _addr(W2), _addr(b2), _addr(W3),
                                    _addr(b3), hidden, classes, _addr(pred), st), None)


def kmeans_init(X, N: int, D: int, K: int, G: int, init_centroids, opt: kmeans_options | None = None):
    """Returns the opaque context handle (an int)."""
    ctx = ctypes.c_void_p()
    rc = lib().kmeans_init(ctypes.byref(ctx), _addr(X), N, D, K, G, _addr(init_centroids),
                           ctypes.byref(opt) if opt is not None else None)
    _check(rc, None)
    return ctx.value


def kmeans_iterate(ctx) -> dict:
    st = kmeans_iter_stats()
    _check(lib().kmeans_iterate(ctx, ctypes.byref(st)), ctx)
    return st.as_dict()


def kmeans_fit(ctx, max_iter: int, tol: float, labels=None, centroids=None, objective=None, n_iter=None):
    """Outputs go to the given arrays (host or device); when ``objective`` /
    ``n_iter`` are None, their values are returned as ``(n_iter, objective)``."""
    J = ctypes.c_double()
    ni = ctypes.c_int32()
    rc = lib().kmeans_fit(ctx, max_iter, tol, _addr(labels), _addr(centroids),
                          _addr(objective) if objective is not None else ctypes.addressof(J),
                          _addr(n_iter) if n_iter is not None else ctypes.addressof(ni))
    _check(rc, ctx)
    return ni.value, J.value


def kmeans_get_labels(ctx, labels) -> None:
    _check(lib().kmeans_get_labels(ctx, _addr(labels)), ctx)


def kmeans_get_centroids(ctx, C) -> None:
    _check(lib().kmeans_get_centroids(ctx, _addr(C)), ctx)


def kmeans_get_stats(ctx, t: int) -> dict:
    st = kmeans_iter_stats()
    _check(lib().kmeans_get_stats(ctx, t, ctypes.byref(st)), ctx)
    return st.as_dict()


def kmeans_get_bounds(ctx, u=None, lbg=None, lb=None) -> None:
    _check(lib().kmeans_get_bounds(ctx, _addr(u), _addr(lbg), _addr(lb)), ctx)


def kmeans_get_groups(ctx, grp=None) -> int:
    """Fills grp (K int32) with each centroid's group; returns the number of groups."""
    n = ctypes.c_int32()
    _check(lib().kmeans_get_groups(ctx, _addr(grp), ctypes.byref(n)), ctx)
    return n.value


def kmeans_get_iteration(ctx) -> int:
    t = ctypes.c_int32()
    _check(lib().kmeans_get_iteration(ctx, ctypes.byref(t)), ctx)
    return t.value


def kmeans_get_kernel_count(ctx) -> int:
    n = ctypes.c_int64()
    _check(lib().kmeans_get_kernel_count(ctx, ctypes.byref(n)), ctx)
    return n.value


def kmeans_reset(ctx, init_centroids) -> None:
    _check(lib().kmeans_reset(ctx, _addr(init_centroids)), ctx)


def kmeans_get_profile(ctx, kind: int):
    """Returns ``(launches, total_ms)`` for one KM_KERNEL_* kind."""
    n = ctypes.c_int64()
    ms = ctypes.c_double()
    _check(lib().kmeans_get_profile(ctx, kind, ctypes.byref(n), ctypes.byref(ms)), ctx)
    return n.value, ms.value


KM_NOALLOC_MAX_K = 1024
KM_NOALLOC_MAX_D = 128


def _check_tensor(name: str, a, dtype: str, shape: tuple) -> None:
    """Raise KMeansError(KM_EINVAL) unless `a` (torch tensor or NumPy array;
    raw addresses are passed through unchecked) has the element type, the
    shape and a C-contiguous layout the C call reads it with."""
    if a is None or isinstance(a, int):
        return
    dt = str(getattr(a, "dtype", "")).replace("torch.", "")
    if dt != dtype:
        raise KMeansError(KM_EINVAL, f"{name} must be {dtype}, got {dt}")
    if tuple(a.shape) != tuple(shape):
        raise KMeansError(KM_EINVAL, f"{name} must have shape {tuple(shape)}, got {tuple(a.shape)}")
    contig = a.is_contiguous() if hasattr(a, "is_contiguous") else a.flags["C_CONTIGUOUS"]
    if not contig:
        raise KMeansError(KM_EINVAL, f"{name} must be C-contiguous")


def kmeans_lloyd_step_noalloc(X, N: int, D: int, C, K: int, labels, C_new, objective, stream=None) -> None:
    """One plain-Lloyd iteration with no allocation (device arrays only;
    stream-ordered, does not wait).  See include/kpynq.h.  Tensors are
    checked for type (float32 X, C, C_new; int32 labels; float64 objective),
    shape and contiguity before the call, since the C side cannot tell."""
    _check_tensor("X", X, "float32", (N, D))
    _check_tensor("C", C, "float32", (K, D))
    _check_tensor("C_new", C_new, "float32", (K, D))
    _check_tensor("labels", labels, "int32", (N,))
    _check_tensor("objective", objective, "float64", (1,))
    st = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    _check(lib().kmeans_lloyd_step_noalloc(_addr(X), N, D, _addr(C), K, _addr(labels), _addr(C_new),
                                           _addr(objective), st), None)


def kmeans_shard_assign(ctx, tol: float, S, Q, cnt) -> int:
    """This shard's assignment and cluster sums (into S, Q, cnt); returns its label changes."""
    nc = ctypes.c_int64()
    _check(lib().kmeans_shard_assign(ctx, tol, _addr(S), _addr(Q), _addr(cnt), ctypes.byref(nc)), ctx)
    return nc.value


def kmeans_shard_update(ctx, final_pass: bool, S, Q, cnt, n_changed: int):
    """The update from the summed statistics; returns (stats dict, objective of a final pass)."""
    st = kmeans_iter_stats()
    J = ctypes.c_double(float("nan"))
    _check(lib().kmeans_shard_update(ctx, int(final_pass), _addr(S), _addr(Q), _addr(cnt), n_changed,
                                     ctypes.byref(st), ctypes.byref(J)), ctx)
    return st.as_dict(), J.value


def kmeans_init_kmeanspp(X, N: int, D: int, K: int, u, centroids, indices=None, stream=None) -> None:
    """k-means++ seeding: K centres of X (device) from the K uniforms u."""
    st = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    _check(lib().kmeans_init_kmeanspp(_addr(X), N, D, K, _addr(u), _addr(centroids), _addr(indices), st), None)


def kmeans_selftest_timeout(polls: int) -> int:
    """The bounded-wait self-test's status (KM_ETIMEOUT expected); does not raise."""
    return lib().kmeans_selftest_timeout(polls)


def kmeans_debug_fail_alloc(after: int) -> None:
    """Make context allocations fail after `after` more (negative: off)."""
    lib().kmeans_debug_fail_alloc(after)


def kmeans_destroy(ctx) -> None:
    if ctx:
        lib().kmeans_destroy(ctx)


def kmeans_last_error(ctx=None) -> str:
    return lib().kmeans_last_error(ctx).decode(errors="replace")


def kmeans_launch_count() -> int:
    return lib().kmeans_launch_count()


# ---------------------------------------------------------------------------
# convenience: a context that owns its handle and keeps its inputs alive
# ---------------------------------------------------------------------------
@dataclass
class FitResult:
    labels: object
    centroids: object
    objective: float
    n_iter: int
    stats: list


class KMeans:
    """One problem on the GPU.  ``X`` / ``C0``: torch tensors (CUDA or CPU) or
    NumPy arrays, float32, row-major.  A CUDA ``X`` is borrowed (kept alive by
    this object)."""

    def __init__(self, X, C0, G: int, *, algo: int = KM_ALGO_FILTERED, stream=None, validate: bool = False,
                 profile: bool = False, dense: int = KM_DENSE_AUTO, dense_switch: float = 0.0,
                 dtype: int | None = None, grouping: int = KM_GROUP_CONTIGUOUS):
        N, D = X.shape
        K = C0.shape[0]
        opt = kmeans_default_options()
        opt.algo = algo
        opt.grouping = grouping
        opt.validate = int(validate)
        opt.profile = int(profile)
        opt.dense = dense
        opt.dense_switch = dense_switch
        opt.dtype = _dtype_of(X, dtype)
        if stream is not None:
            opt.stream = stream if isinstance(stream, int) else stream.cuda_stream
        self._keep = (X, C0)
        self.N, self.D, self.K, self.G = N, D, K, G
        self.ctx = kmeans_init(X, N, D, K, G, C0, opt)

    def set_proposal(self, params: dict | None):
        """params: {"W1", "b1", "W2", "b2", "W3", "b3"} FP32 arrays (host or
        device), or None to remove the proposal."""
        if params is None:
            kmeans_set_proposal(self.ctx, None, None, None, None, None, None, 0)
            self._proposal = None
            return
        w = [params[k] for k in MLP_NAMES]
        self._proposal = w  # keep the arrays alive until the copy has been made
        kmeans_set_proposal(self.ctx, *w, int(w[0].shape[0]))

    def close(self):
        if getattr(self, "ctx", None):
            kmeans_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def groups(self, grp=None) -> int:
        """Number of groups; fills grp (K int32) with each centroid's group."""
        return kmeans_get_groups(self.ctx, grp)

    def reset(self, C0):
        """Restart from new initial centroids (no allocation)."""
        self._keep = (self._keep[0], C0)
        kmeans_reset(self.ctx, C0)

    def profile(self) -> dict:
        """Per kernel kind: (launches, total device ms)."""
        return {KERNEL_KIND_NAMES[k]: kmeans_get_profile(self.ctx, k) for k in range(len(KERNEL_KIND_NAMES))}

    def iterate(self) -> dict:
        return kmeans_iterate(self.ctx)

    def fit(self, max_iter: int, tol: float = 0.0, labels=None, centroids=None, with_stats: bool = True) -> FitResult:
        t0 = kmeans_get_iteration(self.ctx)
        n_iter, J = kmeans_fit(self.ctx, max_iter, tol, labels, centroids)
        stats = self.stats(t0, t0 + n_iter) if with_stats else None
        return FitResult(labels, centroids, J, n_iter, stats)

    def final_stats(self) -> dict:
        """Statistics of the last fit's final assignment (its path, label
        changes, distance evaluations and objective)."""
        return kmeans_get_stats(self.ctx, -1)

    def stats(self, t0: int, t1: int) -> list:
        """Per-iteration statistics of iterations t0 .. t1-1."""
        return [kmeans_get_stats(self.ctx, t) for t in range(t0, t1)]

    def labels(self, out):
        kmeans_get_labels(self.ctx, out)
        return out

    def centroids(self, out):
        kmeans_get_centroids(self.ctx, out)
        return out

    def bounds(self, u=None, lbg=None, lb=None):
        kmeans_get_bounds(self.ctx, u, lbg, lb)
        return u, lbg, lb

    @property
    def iteration(self) -> int:
        return kmeans_get_iteration(self.ctx)

    @property
    def kernel_count(self) -> int:
        return kmeans_get_kernel_count(self.ctx)


def _check_batch(rc: int, b=None):
    if rc != KM_OK:
        msg = lib().kmeans_batch_last_error(b).decode(errors="replace")
        raise KMeansError(rc, msg)


def kmeans_batch_init(problems, opt: kmeans_options, tune_cache: str | None = None):
    """problems: a ctypes array of kmeans_problem.  Returns the batch handle."""
    b = ctypes.c_void_p()
    _check_batch(lib().kmeans_batch_init(ctypes.byref(b), len(problems), problems, ctypes.byref(opt),
                                         tune_cache.encode() if tune_cache else None))
    return b


def kmeans_batch_fit(b, max_iter: int, tol: float) -> None:
    _check_batch(lib().kmeans_batch_fit(b, max_iter, tol), b)


def kmeans_batch_get(b, i: int, labels=None, centroids=None):
    """(objective, iterations of the last fit) of problem i."""
    J = ctypes.c_double()
    n = ctypes.c_int32()
    _check_batch(lib().kmeans_batch_get(b, i, _addr(labels), _addr(centroids), ctypes.byref(J), ctypes.byref(n)), b)
    return J.value, n.value


def kmeans_batch_reset(b) -> None:
    _check_batch(lib().kmeans_batch_reset(b), b)


def kmeans_batch_get_switch(b, i: int) -> float:
    v = ctypes.c_float()
    _check_batch(lib().kmeans_batch_get_switch(b, i, ctypes.byref(v)), b)
    return v.value


def kmeans_batch_get_tuning(b, i: int):
    """(switch, dense engine, survivor queue entries per claim) of problem i."""
    sw, de, gr = ctypes.c_float(), ctypes.c_int32(), ctypes.c_int32()
    _check_batch(lib().kmeans_batch_get_tuning(b, i, ctypes.byref(sw), ctypes.byref(de), ctypes.byref(gr)), b)
    return sw.value, de.value, gr.value


def kmeans_batch_destroy(b) -> None:
    lib().kmeans_batch_destroy(b)


def kmeans_batch_last_error(b=None) -> str:
    return lib().kmeans_batch_last_error(b).decode(errors="replace")


class KMeansBatch:
    """Many independent problems fitted by one CUDA graph launch.

    ``problems``: a list of ``(X, C0, G)`` (N x D and K x D float32 arrays,
    host or device; they must outlive the batch).  ``tune_cache``: path of
    the autotuner's cache file (None: the library's default switch)."""

    def __init__(self, problems, algo: int = KM_ALGO_FILTERED, stream=None, dense: int = KM_DENSE_AUTO,
                 dense_switch: float = 0.0, tune_cache: str | None = None, dtype: int | None = None,
                 grouping: int = KM_GROUP_CONTIGUOUS):
        arr = (kmeans_problem * len(problems))()
        self._keep = []
        for i, (X, C0, G) in enumerate(problems):
            N, D = X.shape
            arr[i] = kmeans_problem(_addr(X), N, D, C0.shape[0], G, _addr(C0))
            self._keep.append((X, C0))
        self.shapes = [(X.shape[0], X.shape[1], C0.shape[0], G) for X, C0, G in problems]
        opt = kmeans_options()
        lib().kmeans_default_options(ctypes.byref(opt))
        opt.algo = algo
        opt.grouping = grouping
        opt.dense = dense
        opt.dense_switch = dense_switch
        opt.dtype = _dtype_of(problems[0][0], dtype) if problems else KM_DTYPE_F32
        if stream is not None:
            opt.stream = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        self.b = kmeans_batch_init(arr, opt, tune_cache)

    def fit(self, max_iter: int, tol: float = 0.0):
        kmeans_batch_fit(self.b, max_iter, tol)

    def reset(self):
        kmeans_batch_reset(self.b)

    def get(self, i: int, labels=None, centroids=None):
        """(objective, iterations) of problem i; fills labels / centroids if given."""
        return kmeans_batch_get(self.b, i, labels, centroids)

    def switch(self, i: int) -> float:
        return kmeans_batch_get_switch(self.b, i)

    def tuning(self, i: int):
        """(switch, dense engine, survivor queue entries per claim) of problem i."""
        return kmeans_batch_get_tuning(self.b, i)

    def close(self):
        if getattr(self, "b", None):
            kmeans_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# the proposal network on the tensor cores (training and inference)
# ---------------------------------------------------------------------------
def _check_mlp(rc: int, m=None):
    if rc != KM_OK:
        msg = lib().kmeans_mlp_last_error(m).decode(errors="replace")
        raise KMeansError(rc, msg)


def kmeans_mlp_create(D: int, hidden: int, classes: int, seed: int = 0, stream=None):
    m = ctypes.c_void_p()
    st = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    _check_mlp(lib().kmeans_mlp_create(ctypes.byref(m), D, hidden, classes, seed, st), None)
    return m.value


def kmeans_mlp_set_params(m, W1, b1, W2, b2, W3, b3) -> None:
    _check_mlp(lib().kmeans_mlp_set_params(m, _addr(W1), _addr(b1), _addr(W2), _addr(b2), _addr(W3), _addr(b3)), m)


def kmeans_mlp_get_params(m, W1=None, b1=None, W2=None, b2=None, W3=None, b3=None) -> None:
    _check_mlp(lib().kmeans_mlp_get_params(m, _addr(W1), _addr(b1), _addr(W2), _addr(b2), _addr(W3), _addr(b3)), m)


def kmeans_mlp_gradient(m, X, y, B: int, grad) -> float:
    """Gradient of the mean cross-entropy on the batch into ``grad``; returns the loss."""
    loss = ctypes.c_double()
    _check_mlp(lib().kmeans_mlp_gradient(m, _addr(X), _addr(y), B, ctypes.byref(loss), _addr(grad)), m)
    return loss.value


def kmeans_mlp_train(m, X, N: int, labels, K: int, steps: int, batch: int, lr: float, seed: int):
    """Adam steps on rows drawn from (X, labels); returns (mean loss, accuracy) over the steps."""
    loss, acc = ctypes.c_double(), ctypes.c_double()
    _check_mlp(lib().kmeans_mlp_train(m, _addr(X), N, _addr(labels), K, steps, batch, lr, seed,
                                      ctypes.byref(loss), ctypes.byref(acc)), m)
    return loss.value, acc.value


def kmeans_mlp_predict_net(m, X, N: int, pred) -> None:
    _check_mlp(lib().kmeans_mlp_predict_net(m, _addr(X), N, _addr(pred)), m)


def kmeans_mlp_destroy(m) -> None:
    if m:
        lib().kmeans_mlp_destroy(m)


def kmeans_mlp_last_error(m=None) -> str:
    return lib().kmeans_mlp_last_error(m).decode(errors="replace")


class MLP:
    """The proposal network D -> hidden -> hidden -> classes (GELU), trained
    and evaluated on the tensor cores.  Parameters are exchanged as FP32
    arrays with O3's names and shapes (W1 hidden x D, b1, W2, b2, W3 classes x
    hidden, b3)."""

    def __init__(self, D: int, hidden: int, classes: int, seed: int = 0, stream=None):
        self.D, self.H, self.G = D, hidden, classes
        self.m = kmeans_mlp_create(D, hidden, classes, seed, stream)

    def shapes(self) -> dict:
        D, H, G = self.D, self.H, self.G
        return {"W1": (H, D), "b1": (H,), "W2": (H, H), "b2": (H,), "W3": (G, H), "b3": (G,)}

    def n_params(self) -> int:
        n = 0
        for shp in self.shapes().values():
            k = 1
            for v in shp:
                k *= v
            n += k
        return n

    def split(self, vec) -> dict:
        """A flat parameter-layout vector as a dict of views with O3's names."""
        out, o = {}, 0
        for k, shp in self.shapes().items():
            n = 1
            for v in shp:
                n *= v
            out[k] = vec[o:o + n].reshape(shp)
            o += n
        return out

    def set_params(self, params: dict) -> None:
        w = [params[k] for k in MLP_NAMES]
        kmeans_mlp_set_params(self.m, *w)

    def get_params(self, out: dict) -> dict:
        kmeans_mlp_get_params(self.m, *[out[k] for k in MLP_NAMES])
        return out

    def gradient(self, X, y, grad) -> float:
        return kmeans_mlp_gradient(self.m, X, y, X.shape[0], grad)

    def train(self, X, labels, K: int, steps: int, batch: int = 8192, lr: float = 1e-3, seed: int = 1):
        return kmeans_mlp_train(self.m, X, X.shape[0], labels, K, steps, batch, lr, seed)

    def predict(self, X, pred):
        kmeans_mlp_predict_net(self.m, X, X.shape[0], pred)
        return pred

    def close(self):
        if getattr(self, "m", None):
            kmeans_mlp_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
