"""FP64 CPU oracle for triangle-inequality K-means -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package.  The product library
(``paper_1905_09345_gb300``) never imports it, and it imports nothing from the
product; the two share only the seeded input generators, which hold none of the
method's arithmetic.

Two independent C implementations, each written from its definition:

* ``lloyd.c`` (O1): brute-force Lloyd -- the plain definition of the result
  KPynq's filters must reproduce exactly (Abstract; Sec. I: the filters only
  remove distance computations).
* ``ti_lloyd.c`` (O2): the filtered method step by step (global / group-level
  filter, point-level filter, distance calculator, bound refresh; Sec. I), in
  FP64, with per-iteration skip counters.

* ``kmeanspp.c`` (O4): k-means++ seeding (D^2 sampling) with the random
  numbers as inputs and an exactly reproducible draw -- an initialisation the
  library offers beside the caller's centroids (the paper takes them as given).

* ``mlp.py`` (O3): the learned group proposal's MLP (GELU layers, softmax
  cross-entropy, Adam) in numpy FP64 -- a layered form of the library, not in
  the paper; the filtered method's labels do not depend on it.

Groupings for O2: ``contiguous_groups`` (centroid j -> group floor(jG/K)) and
``clustered_groups`` (Lloyd over the centroids, seeded by their first G rows);
the paper does not say how groups form, and labels do not depend on it.

Pins (``tests/test_oracle_*.py``, ``-m "not gpu"``): closed forms (K = 1 mean,
K = N zero objective), a hand-derived worked example (``tests/golden``),
scipy ``cdist`` and scikit-learn's Lloyd as independent library routines,
Lloyd invariants (monotone objective, fixed point), exact tie cases, O2 == O1
label-for-label every iteration (under contiguous, clustered, random and
partly empty groupings), O2 bound validity, O2's per-iteration skip counters
against hand-derived traces (``tests/golden/o2_filter_counts.json``), the
clustered grouping's fixed point and degenerate cases, and planted mistakes
that the pins must catch (one per skip counter among them).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_SOURCES = {"lloyd": "lloyd.c", "ti": "ti_lloyd.c", "pp": "kmeanspp.c"}
_lock = threading.Lock()
_libs: dict = {}

# O2 counter layout (CNT_* in ti_lloyd.c)
CNT_GLOBAL, CNT_TIGHT, CNT_GROUP, CNT_POINT, CNT_DIST, CNT_CHANGED = range(6)
CNT_N = 6


def _lib_path(name: str) -> str:
    return os.path.join(_LIBDIR, f"liboracle_{name}.so")


def _compile(src: str, out: str) -> None:
    os.makedirs(os.path.dirname(out), exist_ok=True)
    base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=c11"]
    tmp = out + f".tmp{os.getpid()}"
    # OpenMP only splits independent per-point work; fall back without it.
    for extra in (["-fopenmp"], []):
        r = subprocess.run(base + extra + [src, "-o", tmp, "-lm"],
                           capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, out)
            return
    raise RuntimeError(f"oracle build failed for {src}:\n{r.stderr}")


def build(force: bool = False) -> None:
    """Compile both oracle libraries with gcc (a second or two)."""
    for name, src in _SOURCES.items():
        out = _lib_path(name)
        srcp = os.path.join(_HERE, src)
        if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(srcp):
            _compile(srcp, out)


def _load(name: str, lib=None):
    if lib is not None:
        return lib
    with _lock:
        if name in _libs:
            return _libs[name]
        srcp = os.path.join(_HERE, _SOURCES[name])
        path = _lib_path(name)
        if not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(srcp):
            _compile(srcp, path)
        lib = ctypes.CDLL(path)
        _declare(lib, name)
        _libs[name] = lib
        return lib


def compile_variant(name: str, replacements, workdir: str):
    """Compile a copy of oracle source ``name`` ("lloyd" or "ti") with textual
    ``(old, new)`` replacements applied -- used only by the tests that plant a
    mistake in the oracle and check that a pin catches it.  Returns the
    loaded library, to be passed as ``lib=`` to the wrapper functions."""
    with open(os.path.join(_HERE, _SOURCES[name])) as f:
        src = f.read()
    for old, new in replacements:
        if old not in src:
            raise ValueError(f"mutation anchor not found: {old!r}")
        src = src.replace(old, new, 1)
    tag = abs(hash(tuple(replacements))) % (1 << 40)
    cpath = os.path.join(workdir, f"{name}_{tag}.c")
    with open(cpath, "w") as f:
        f.write(src)
    out = os.path.join(workdir, f"lib{name}_{tag}.so")
    _compile(cpath, out)
    lib = ctypes.CDLL(out)
    _declare(lib, name)
    return lib


_dp = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_lp = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_i64, _i32, _f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
_vp = ctypes.c_void_p


def _declare(lib, name: str) -> None:
    if name == "lloyd":
        lib.o1_assign.restype = _i64
        lib.o1_assign.argtypes = [_dp, _i64, _i32, _dp, _i32, _vp, _ip, _vp, _vp]
        lib.o1_objective.restype = _f64
        lib.o1_objective.argtypes = [_dp, _i64, _i32, _ip, _dp, _i32]
        lib.o1_update.restype = _f64
        lib.o1_update.argtypes = [_dp, _i64, _i32, _ip, _dp, _i32, _dp, _vp]
        lib.o1_fit.restype = _i32
        lib.o1_fit.argtypes = [_dp, _i64, _i32, _dp, _i32, _i32, _f64, _ip, _dp,
                               _vp, _vp, _vp]
    elif name == "pp":
        lib.o4_kmeanspp.restype = _i32
        lib.o4_kmeanspp.argtypes = [_dp, _i64, _i32, _i32, _dp, _lp, _vp]
    else:
        lib.o2_init_assign.restype = None
        lib.o2_init_assign.argtypes = [_dp, _i64, _i32, _dp, _i32, _i32, _ip, _ip,
                                       _dp, _dp, _lp]
        lib.o2_assign.restype = None
        lib.o2_assign.argtypes = [_dp, _i64, _i32, _dp, _i32, _i32, _ip, _dp, _dp,
                                  _ip, _dp, _dp, _lp]
        lib.o2_update.restype = _f64
        lib.o2_update.argtypes = [_dp, _i64, _i32, _ip, _dp, _i32, _i32, _ip, _dp,
                                  _dp, _dp]
        lib.o2_fit.restype = _i32
        lib.o2_fit.argtypes = [_dp, _i64, _i32, _dp, _i32, _i32, _ip, _i32, _f64,
                               _ip, _dp, _vp, _vp, _vp, _vp]


def _as64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def contiguous_groups(K: int, G: int) -> np.ndarray:
    """Centroid j -> group floor(j * G / K): balanced, deterministic grouping."""
    return ((np.arange(K, dtype=np.int64) * G) // K).astype(np.int32)


def clustered_groups(C, G: int, iters: int = 5) -> np.ndarray:
    """The clustered grouping (the Yinyang-style reading of how groups form;
    the paper does not say): Lloyd's algorithm over the K centroids
    themselves, in FP64, seeded with their first G rows, for ``iters``
    iterations; centroid k joins the group whose centre is nearest (lowest
    index on ties) after the last update.  An empty group keeps its centre.
    Labels of the filtered method do not depend on the grouping; only how
    much the filters skip does."""
    C = _as64(C)
    K = C.shape[0]
    if not 1 <= G <= K:
        raise ValueError("need 1 <= G <= K")
    centres = C[:G].copy()
    grp = np.zeros(K, np.int32)
    for it in range(iters + 1):
        d = ((C[:, None, :] - centres[None, :, :]) ** 2).sum(axis=2)
        grp = np.argmin(d, axis=1).astype(np.int32)  # first minimum: lowest index
        if it == iters:
            break
        for g in range(G):
            m = grp == g
            if m.any():
                centres[g] = C[m].mean(axis=0)
    return grp


# ----------------------------------------------------------------------------
# O1: brute-force Lloyd
# ----------------------------------------------------------------------------
def lloyd_assign(X, C, prev=None, *, lib=None):
    """Nearest centroid per point (lowest index on ties).

    Returns ``(labels, d1sq, d2sq, n_changed)``: the label, the smallest and
    second-smallest squared distances (FP64), and the number of labels that
    differ from ``prev`` (N when ``prev`` is None).
    """
    lib = _load("lloyd", lib)
    X, C = _as64(X), _as64(C)
    N, D = X.shape
    K = C.shape[0]
    labels = np.empty(N, np.int32)
    d1 = np.empty(N, np.float64)
    d2 = np.empty(N, np.float64)
    pv = None if prev is None else np.ascontiguousarray(prev, dtype=np.int32)
    ch = lib.o1_assign(X, N, D, C, K, _ptr(pv), labels, _ptr(d1), _ptr(d2))
    return labels, d1, d2, int(ch)


def lloyd_update(X, labels, C_old, *, lib=None):
    """Centroid means (empty cluster keeps ``C_old``).  Returns ``(C_new, counts, J)``
    with ``J = J(labels, C_old)``."""
    lib = _load("lloyd", lib)
    X, C_old = _as64(X), _as64(C_old)
    N, D = X.shape
    K = C_old.shape[0]
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    C_new = np.empty_like(C_old)
    counts = np.empty(K, np.int64)
    J = lib.o1_update(X, N, D, labels, C_old, K, C_new, _ptr(counts))
    return C_new, counts, float(J)


def lloyd_objective(X, labels, C, *, lib=None) -> float:
    lib = _load("lloyd", lib)
    X, C = _as64(X), _as64(C)
    N, D = X.shape
    return float(lib.o1_objective(X, N, D, np.ascontiguousarray(labels, dtype=np.int32),
                                  C, C.shape[0]))


def lloyd_fit(X, C0, max_iter: int, tol: float = 0.0, *, lib=None) -> dict:
    """Full brute-force Lloyd run.  Keys: labels, centroids, objective, n_iter,
    J_hist, changed_hist."""
    lib = _load("lloyd", lib)
    X, C0 = _as64(X), _as64(C0)
    N, D = X.shape
    K = C0.shape[0]
    labels = np.empty(N, np.int32)
    C = np.empty_like(C0)
    Jh = np.zeros(max(max_iter, 1), np.float64)
    ch = np.zeros(max(max_iter, 1), np.int64)
    Jf = np.zeros(1, np.float64)
    n_iter = lib.o1_fit(X, N, D, C0, K, max_iter, tol, labels, C, _ptr(Jh), _ptr(ch), _ptr(Jf))
    if n_iter < 0:
        raise MemoryError("oracle allocation failed")
    return dict(labels=labels, centroids=C, objective=float(Jf[0]), n_iter=int(n_iter),
                J_hist=Jh[:n_iter].copy(), changed_hist=ch[:n_iter].copy())


# ----------------------------------------------------------------------------
# O2: triangle-inequality filtered K-means
# ----------------------------------------------------------------------------
class TIState:
    """Step-by-step access to the filtered oracle (for bound-invariant tests)."""

    def __init__(self, X, C0, G: int, grp=None, *, lib=None):
        self.lib = _load("ti", lib)
        self.X = _as64(X)
        self.N, self.D = self.X.shape
        self.C = _as64(C0).copy()
        self.K = self.C.shape[0]
        self.G = G
        self.grp = (contiguous_groups(self.K, G) if grp is None
                    else np.ascontiguousarray(grp, dtype=np.int32))
        self.a = np.zeros(self.N, np.int32)
        self.u = np.zeros(self.N, np.float64)
        self.lb = np.zeros((self.N, G), np.float64)
        self.delta = np.zeros(self.K, np.float64)
        self.delta_g = np.zeros(G, np.float64)
        self.cnt = np.zeros(CNT_N, np.int64)
        self.t = 0

    def assign(self):
        """Assignment from the current centroids; updates a, u, lb, cnt."""
        if self.t == 0:
            self.lib.o2_init_assign(self.X, self.N, self.D, self.C, self.K, self.G,
                                    self.grp, self.a, self.u, self.lb, self.cnt)
        else:
            self.lib.o2_assign(self.X, self.N, self.D, self.C, self.K, self.G, self.grp,
                               self.delta, self.delta_g, self.a, self.u, self.lb, self.cnt)
        return self.cnt.copy()

    def update(self) -> float:
        """Centroid update + drift; returns J(a, C_old) and advances t."""
        C_new = np.empty_like(self.C)
        J = self.lib.o2_update(self.X, self.N, self.D, self.a, self.C, self.K, self.G,
                               self.grp, C_new, self.delta, self.delta_g)
        self.C = C_new
        self.t += 1
        return float(J)


def ti_fit(X, C0, G: int, max_iter: int, tol: float = 0.0, grp=None, *,
           keep_history: bool = True, lib=None) -> dict:
    """Full filtered run (same stopping rule as :func:`lloyd_fit`).  Keys:
    labels, centroids, objective, n_iter, J_hist, cnt_hist (n_iter x CNT_N),
    labels_hist (n_iter x N, if ``keep_history``)."""
    lib = _load("ti", lib)
    X, C0 = _as64(X), _as64(C0)
    N, D = X.shape
    K = C0.shape[0]
    grp = contiguous_groups(K, G) if grp is None else np.ascontiguousarray(grp, dtype=np.int32)
    labels = np.empty(N, np.int32)
    C = np.empty_like(C0)
    m = max(max_iter, 1)
    lh = np.zeros((m, N), np.int32) if keep_history else None
    Jh = np.zeros(m, np.float64)
    cnt = np.zeros((m, CNT_N), np.int64)
    Jf = np.zeros(1, np.float64)
    n_iter = lib.o2_fit(X, N, D, C0, K, G, grp, max_iter, tol, labels, C,
                        _ptr(lh), _ptr(Jh), _ptr(cnt), _ptr(Jf))
    if n_iter < 0:
        raise MemoryError("oracle allocation failed")
    out = dict(labels=labels, centroids=C, objective=float(Jf[0]), n_iter=int(n_iter),
               J_hist=Jh[:n_iter].copy(), cnt_hist=cnt[:n_iter].copy())
    if keep_history:
        out["labels_hist"] = lh[:n_iter].copy()
    return out


# ----------------------------------------------------------------------------
# O4: k-means++ seeding
# ----------------------------------------------------------------------------
def kmeanspp(X, K: int, u, *, lib=None):
    """k-means++ centre indices (O4, ``kmeanspp.c``): ``u`` holds K uniforms
    in [0, 1), one per centre.  Returns ``(idx int64 (K,), dmin (N,))``, dmin
    the final squared distance of every point to its nearest chosen centre."""
    lib = _load("pp", lib)
    X = _as64(X)
    N, D = X.shape
    u = _as64(u)
    if u.shape != (K,):
        raise ValueError("u must hold K uniforms")
    idx = np.empty(K, np.int64)
    dmin = np.empty(N, np.float64)
    if lib.o4_kmeanspp(X, N, D, K, u, idx, _ptr(dmin)) != 0:
        raise ValueError("bad arguments or allocation failure")
    return idx, dmin


# ----------------------------------------------------------------------------
# near-tie classification (the parity rule for GPU labels)
# ----------------------------------------------------------------------------
NEAR_TIE_REL = 1e-6


def near_ties(d1sq, d2sq, rel: float = NEAR_TIE_REL) -> np.ndarray:
    """True where the FP64 gap between the two nearest centroids, in
    Euclidean distance, is at most ``rel`` times the second distance
    (d2 = 0 counts as a near-tie)."""
    d1 = np.sqrt(np.asarray(d1sq, np.float64))
    d2 = np.sqrt(np.asarray(d2sq, np.float64))
    return (d2 - d1) <= rel * d2
