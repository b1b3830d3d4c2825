"""Seeded synthetic inputs: Gaussian mixtures shaped like the paper's workloads.

KPynq evaluates on six UCI datasets it does not name, "covering a wide range of
size and dimensionality" (Sec. II).  They are not available here; these seeded
Gaussian mixtures stand in for them, at the sizes of the five workloads this
library is measured on.  This module holds input generation only -- none of the
K-means arithmetic -- and is the one piece of code that both the CUDA path's
tests/benchmark and the CPU oracle are fed from.

All draws use ``numpy.random.default_rng(seed)`` (PCG64) in a fixed order:
blob centres, blob scales, mixture counts, per-point noise, the shuffle, then
the initial-centroid sample.  Data is produced in float32 (the library's input
type); ``to_bf16`` rounds a float32 array to bfloat16 storage values.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    """One synthetic K-means problem."""
    name: str
    X: np.ndarray            # (N, D) float32, row-major
    C0: np.ndarray           # (K, D) float32 initial centroids
    G: int                   # number of centroid groups
    max_iter: int
    tol: float
    blob: np.ndarray = field(repr=False, default=None)  # generating blob per point
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return self.X.shape[0]

    @property
    def D(self) -> int:
        return self.X.shape[1]

    @property
    def K(self) -> int:
        return self.C0.shape[0]


def gaussian_mixture(rng: np.random.Generator, N: int, D: int, n_blobs: int, *,
                     centre_range: float, scale: str, scale_args=(), weights: str = "equal",
                     chunk: int = 1 << 20):
    """Draw N points from an ``n_blobs`` Gaussian mixture in D dimensions.

    centres ~ U[-centre_range, centre_range]^D.  ``scale`` selects the blob
    standard deviations: ``"fixed"`` (one value, isotropic), ``"axis_uniform"``
    (per blob and axis, U[lo, hi]: anisotropic), ``"blob_uniform"`` (per blob,
    U[lo, hi], isotropic) or ``"blob_lognormal"`` (per blob, lognormal(mu, s),
    isotropic).  ``weights``: ``"equal"`` (counts as even as N allows) or
    ``"dirichlet"`` (Dirichlet(1) weights, then multinomial counts).
    Returns ``(X float32 (N, D), blob int32 (N,))`` with rows shuffled.
    """
    centres = rng.uniform(-centre_range, centre_range, size=(n_blobs, D)).astype(np.float32)
    if scale == "fixed":
        sig = np.full((n_blobs, 1), scale_args[0], np.float32)
    elif scale == "axis_uniform":
        sig = rng.uniform(scale_args[0], scale_args[1], size=(n_blobs, D)).astype(np.float32)
    elif scale == "blob_uniform":
        sig = rng.uniform(scale_args[0], scale_args[1], size=(n_blobs, 1)).astype(np.float32)
    elif scale == "blob_lognormal":
        sig = rng.lognormal(scale_args[0], scale_args[1], size=(n_blobs, 1)).astype(np.float32)
    else:
        raise ValueError(scale)
    if weights == "equal":
        counts = np.full(n_blobs, N // n_blobs, np.int64)
        counts[: N % n_blobs] += 1
    elif weights == "dirichlet":
        counts = rng.multinomial(N, rng.dirichlet(np.ones(n_blobs)))
    else:
        raise ValueError(weights)
    blob = np.repeat(np.arange(n_blobs, dtype=np.int32), counts)
    X = np.empty((N, D), np.float32)
    for s in range(0, N, chunk):
        e = min(N, s + chunk)
        b = blob[s:e]
        X[s:e] = centres[b] + rng.standard_normal((e - s, D), dtype=np.float32) * sig[b]
    perm = rng.permutation(N)
    return X[perm], blob[perm]


def sample_init(rng: np.random.Generator, X: np.ndarray, K: int) -> np.ndarray:
    """K distinct rows of X, chosen with ``rng.choice(N, K, replace=False)``."""
    idx = rng.choice(X.shape[0], K, replace=False)
    return np.ascontiguousarray(X[idx])


def to_bf16(a: np.ndarray) -> np.ndarray:
    """float32 -> nearest bfloat16 value (ties to even), returned as float32.
    A storage-format conversion of the input, not part of the method."""
    a = np.ascontiguousarray(a, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32)
    return np.where(np.isnan(a), a, out)


def bf16_bits(a: np.ndarray) -> np.ndarray:
    """The uint16 bfloat16 bit patterns of ``to_bf16(a)`` (storage format)."""
    return (to_bf16(a).view(np.uint32) >> 16).astype(np.uint16)


# ---------------------------------------------------------------------------
# the five measured workloads (sizes can be reduced for tests)
# ---------------------------------------------------------------------------
def small_blobs(N: int = 16384, D: int = 16, K: int = 16, G: int = 2, seed: int = 0) -> Workload:
    """Plain filtered K-means, FP32: N=16,384, D=16, K=16, G=2; K isotropic
    blobs, centres U[-10,10]^D, std 1, equal weights; C0 = the first K points;
    20 iterations."""
    rng = np.random.default_rng(seed)
    X, blob = gaussian_mixture(rng, N, D, K, centre_range=10.0, scale="fixed", scale_args=(1.0,))
    return Workload("blobs16k_d16_k16_g2", X, np.ascontiguousarray(X[:K]), G, 20, 0.0, blob,
                    dict(seed=seed))


def anisotropic_1m(N: int = 1 << 20, D: int = 64, K: int = 256, G: int = 26, seed: int = 2) -> Workload:
    """Large FP32 workload: N=1,048,576, D=64, K=256, G=26; 256 anisotropic
    blobs, centres U[-20,20]^D, per-axis std U[0.5,2.0], Dirichlet(1) mixture
    weights; C0 = K points sampled with the data seed; 50 iterations or
    tol 1e-4."""
    rng = np.random.default_rng(seed)
    X, blob = gaussian_mixture(rng, N, D, K, centre_range=20.0, scale="axis_uniform",
                               scale_args=(0.5, 2.0), weights="dirichlet")
    C0 = sample_init(rng, X, K)
    return Workload(f"aniso_n{N}_d{D}_k{K}_g{G}", X, C0, G, 50, 1e-4, blob, dict(seed=seed))


def highdim_4m(N: int = 1 << 22, D: int = 128, K: int = 1024, G: int = 103, seed: int = 3) -> Workload:
    """High-dimension workload: N=4,194,304, D=128, K=1024, G=103; 1024
    isotropic blobs with lognormal(0, 0.5) stds, centres U[-20,20]^D, equal
    weights; stored as bfloat16 values; 30 iterations."""
    rng = np.random.default_rng(seed)
    X, blob = gaussian_mixture(rng, N, D, K, centre_range=20.0, scale="blob_lognormal",
                               scale_args=(0.0, 0.5))
    X = to_bf16(X)
    C0 = sample_init(rng, X, K)
    return Workload(f"highdim_n{N}_d{D}_k{K}_g{G}", X, C0, G, 30, 0.0, blob,
                    dict(seed=seed, storage="bf16"))


def proposal_family(sample_seed: int, N: int = 1 << 23, D: int = 32, K: int = 4096, G: int = 410,
                    family_seed: int = 5) -> Workload:
    """Learned-proposal workload: N=8,388,608, D=32, K=4096, G=410; 4096
    isotropic blobs with std U[0.3,1.5], centres U[-20,20]^D, equal weights.
    The family (centres, stds, C0) is fixed by ``family_seed``; ``sample_seed``
    only redraws the N points.  40 iterations."""
    frng = np.random.default_rng(family_seed)
    centres = frng.uniform(-20.0, 20.0, size=(K, D)).astype(np.float32)
    sig = frng.uniform(0.3, 1.5, size=(K, 1)).astype(np.float32)
    c0_blob = frng.integers(0, K, size=K)
    C0 = (centres[c0_blob] + frng.standard_normal((K, D), dtype=np.float32) * sig[c0_blob])
    rng = np.random.default_rng(sample_seed)
    counts = np.full(K, N // K, np.int64)
    counts[: N % K] += 1
    blob = np.repeat(np.arange(K, dtype=np.int32), counts)
    X = np.empty((N, D), np.float32)
    chunk = 1 << 20
    for s in range(0, N, chunk):
        e = min(N, s + chunk)
        b = blob[s:e]
        X[s:e] = centres[b] + rng.standard_normal((e - s, D), dtype=np.float32) * sig[b]
    perm = rng.permutation(N)
    return Workload(f"proposal_n{N}_d{D}_k{K}_g{G}_s{sample_seed}", X[perm],
                    np.ascontiguousarray(C0, np.float32), G, 40, 0.0, blob[perm],
                    dict(family_seed=family_seed, sample_seed=sample_seed))


def skewed_mixture(N: int = 1 << 20, D: int = 32, K: int = 128, G: int = 13, seed: int = 6) -> Workload:
    """Real-data-like skew (the paper's datasets are raw UCI tables of "a wide
    range of size and dimensionality", Sec. II): K anisotropic blobs with
    power-law sizes (weights proportional to rank^-1.2), features on scales
    spread over three orders of magnitude (per-feature scale lognormal(0,
    1.5)) around per-feature offsets up to 1000 scales, one feature in eight
    rounded to integers (count-like attributes), 1% uniform outliers over the
    bounding box and 2% exact duplicates of other rows.  Initial centroids:
    k-means++ with the uniforms ``meta["pp_u"]`` (drawn after the data); C0
    holds the first K rows until they are computed.  30 iterations or tol 1e-4."""
    rng = np.random.default_rng(seed)
    fscale = rng.lognormal(0.0, 1.5, size=D).astype(np.float32)
    offset = (rng.uniform(0.0, 1000.0, size=D) * fscale).astype(np.float32)
    centres = rng.uniform(-20.0, 20.0, size=(K, D)).astype(np.float32)
    sig = rng.uniform(0.2, 2.0, size=(K, D)).astype(np.float32)
    w = np.arange(1, K + 1, dtype=np.float64) ** -1.2
    counts = rng.multinomial(N, w / w.sum())
    blob = np.repeat(np.arange(K, dtype=np.int32), counts)
    X = np.empty((N, D), np.float32)
    chunk = 1 << 20
    for a in range(0, N, chunk):
        b = min(N, a + chunk)
        bb = blob[a:b]
        X[a:b] = centres[bb] + rng.standard_normal((b - a, D), dtype=np.float32) * sig[bb]
    n_out = N // 100
    lo, hi = X.min(axis=0), X.max(axis=0)
    out_rows = rng.choice(N, n_out, replace=False)
    X[out_rows] = rng.uniform(lo, hi, size=(n_out, D)).astype(np.float32)
    blob[out_rows] = -1
    X = X * fscale + offset
    ints = np.arange(D) % 8 == 7
    X[:, ints] = np.round(X[:, ints])
    n_dup = N // 50
    dst = rng.choice(N, n_dup, replace=False)
    src = rng.choice(N, n_dup, replace=True)
    X[dst] = X[src]
    blob[dst] = blob[src]
    perm = rng.permutation(N)
    X = np.ascontiguousarray(X[perm])
    u = rng.uniform(size=K)
    return Workload(f"skewed_n{N}_d{D}_k{K}_g{G}", X, np.ascontiguousarray(X[:K]), G, 30, 1e-4, blob[perm],
                    dict(seed=seed, pp_u=u, init="kmeans++"))


def batched_problems(n_problems: int = 512, seed0: int = 0, n_lo: int = 1000, n_hi: int = 200000,
                     k_lo: int = 8, k_hi: int = 512):
    """Parameters of the batched workload: per problem p (seed0 + p),
    N ~ logU[n_lo, n_hi], D ~ U{8,32,64,128}, K ~ logU[k_lo, k_hi] (integer,
    at most N), G = max(1, K // 10).  Returns a list of dicts; data comes from
    :func:`batched_problem`."""
    out = []
    for p in range(n_problems):
        rng = np.random.default_rng(seed0 + p)
        N = int(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
        D = int(rng.choice([8, 32, 64, 128]))
        K = int(np.exp(rng.uniform(np.log(k_lo), np.log(k_hi))))
        K = max(1, min(K, N))
        out.append(dict(seed=seed0 + p, N=N, D=D, K=K, G=max(1, K // 10)))
    return out


def batched_problem(spec: dict) -> Workload:
    """One batched problem: K isotropic blobs, centres U[-10,10]^D, std 1,
    equal weights; C0 = the first K points; 25 iterations."""
    rng = np.random.default_rng(10_000 + spec["seed"])
    X, blob = gaussian_mixture(rng, spec["N"], spec["D"], spec["K"], centre_range=10.0,
                               scale="fixed", scale_args=(1.0,))
    return Workload(f"batch{spec['seed']}", X, np.ascontiguousarray(X[: spec["K"]]), spec["G"],
                    25, 0.0, blob, dict(spec))
