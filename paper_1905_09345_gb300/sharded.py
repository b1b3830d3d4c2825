"""Point sharding: one K-means problem split by rows across processes.

Each process (one per GPU) holds a contiguous block of the rows, its own
context over them, and the same initial centroids.  Per iteration the only
exchange is one all-reduce of the cluster statistics (FP64 sums and squared
distances about the current centroids, counts, label changes); every process
then runs the same update on the same sums, so the centroids, drifts and
stop decision agree everywhere and the filters' per-point bounds never leave
their process.  The arithmetic stays in the library (kmeans_shard_assign /
kmeans_shard_update); this module only splits the rows and moves the
statistics through the caller's collective (NCCL for device tensors, gloo
for host tensors).
"""
from __future__ import annotations

from dataclasses import dataclass

from . import kpynq


def shard_rows(N: int, world: int, rank: int) -> tuple[int, int]:
    """Rows [start, stop) of `rank` out of `world`: contiguous blocks whose
    sizes differ by at most one (the first N % world ranks take one more)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need world >= 1 and 0 <= rank < world")
    base, extra = divmod(N, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


class ShardStats:
    """The exchanged statistics of one assignment: an FP64 block [S (K x D) |
    Q (K)] and an int64 block [cnt (K) | n_changed], summed over the shards
    by two in-place all-reduces."""

    def __init__(self, K: int, D: int, device=None):
        import torch
        self.K, self.D = K, D
        self.f = torch.zeros(K * D + K, dtype=torch.float64, device=device)
        self.i = torch.zeros(K + 1, dtype=torch.int64, device=device)

    @property
    def S(self):
        return self.f[: self.K * self.D]

    @property
    def Q(self):
        return self.f[self.K * self.D:]

    @property
    def cnt(self):
        return self.i[: self.K]

    def set_changed(self, n: int) -> None:
        self.i[self.K] = n

    @property
    def changed(self) -> int:
        return int(self.i[self.K].item())

    def allreduce(self, reduce_sum) -> None:
        """reduce_sum(tensor) sums the tensor over all shards in place
        (torch.distributed.all_reduce, or the identity for one shard)."""
        reduce_sum(self.f)
        reduce_sum(self.i)


@dataclass
class ShardFit:
    labels: object       # this shard's labels (device int32)
    centroids: object    # K x D float32 (device), the same on every shard
    objective: float     # J of the final assignment, summed over the shards
    n_iter: int
    stats: list          # per-iteration statistics (global n_changed, J_t; local counters)


def fit_sharded(X, C0, G: int, max_iter: int, tol: float, reduce_sum, *, algo: int = kpynq.KM_ALGO_FILTERED,
                stream=None, exchange_device=None) -> ShardFit:
    """Fit one problem whose rows are split across processes.  X: this
    shard's rows (N_local x D float32, on this process's GPU); C0: the common
    initial centroids; reduce_sum: an in-place sum over the shards.  Returns
    this shard's labels and the common centroids and objective."""
    import torch
    N, D = X.shape
    K = C0.shape[0]
    km = kpynq.KMeans(X, C0, G, algo=algo, stream=stream)
    st = ShardStats(K, D, device=exchange_device)
    stats = []
    n_iter = 0
    try:
        for _ in range(max_iter):
            st.set_changed(kpynq.kmeans_shard_assign(km.ctx, tol, st.S, st.Q, st.cnt))
            st.allreduce(reduce_sum)
            s, _ = kpynq.kmeans_shard_update(km.ctx, False, st.S, st.Q, st.cnt, st.changed)
            stats.append(s)
            n_iter += 1
            if s["done"]:
                break
        # the final assignment to the returned centroids
        st.set_changed(kpynq.kmeans_shard_assign(km.ctx, tol, st.S, st.Q, st.cnt))
        st.allreduce(reduce_sum)
        _, J = kpynq.kmeans_shard_update(km.ctx, True, st.S, st.Q, st.cnt, st.changed)
        dev = X.device if hasattr(X, "device") else None
        labels = torch.empty(N, dtype=torch.int32, device=dev)
        C = torch.empty(K, D, dtype=torch.float32, device=dev)
        km.labels(labels)
        km.centroids(C)
    finally:
        km.close()
    return ShardFit(labels, C, J, n_iter, stats)
