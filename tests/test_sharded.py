"""Point sharding (one problem split by rows across processes).

CPU (gloo, two spawned ranks, no GPU): the row split and the exchange of the
cluster statistics -- each rank's block sums to the totals, counts and label
changes stay integers.  GPU (gloo, two spawned ranks on the one GPU,
host-side exchange between kernels, no kernel waits on another process): the
sharded fit equals the single-process fit -- same iterations, labels equal to
the oracle's FP64 argmin over the common centroids, centroids within 1e-5 of
the single fit's and objective within 1e-9 of the oracle's.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1905_09345_gb300 import sharded  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_rows_cover_and_balance():
    for N in (1, 7, 10, 1 << 20):
        for world in (1, 2, 3, 8):
            blocks = [sharded.shard_rows(N, world, r) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == N
            assert all(a[1] == b[0] for a, b in zip(blocks, blocks[1:]))
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        sharded.shard_rows(10, 2, 2)


def _exchange_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        K, D = 5, 3
        st = sharded.ShardStats(K, D)
        rng = np.random.default_rng(rank)
        S = rng.normal(size=K * D)
        Q = rng.uniform(size=K)
        cnt = rng.integers(0, 1000, K)
        st.S.copy_(torch.from_numpy(S))
        st.Q.copy_(torch.from_numpy(Q))
        st.cnt.copy_(torch.from_numpy(cnt))
        st.set_changed(7 + rank)
        st.allreduce(lambda t: dist.all_reduce(t, op=dist.ReduceOp.SUM))
        out.put((rank, st.S.numpy().copy(), st.Q.numpy().copy(), st.cnt.numpy().copy(), st.changed))
    finally:
        dist.destroy_process_group()


def test_exchange_sums_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_exchange_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    K, D = 5, 3
    want_S = sum(np.random.default_rng(r).normal(size=K * D) for r in range(2))
    for rank, S, Q, cnt, ch in got:
        rs = [np.random.default_rng(r) for r in range(2)]
        parts = [(g.normal(size=K * D), g.uniform(size=K), g.integers(0, 1000, K)) for g in rs]
        assert np.allclose(S, want_S, rtol=0, atol=1e-15)
        assert np.allclose(Q, parts[0][1] + parts[1][1], rtol=0, atol=1e-15)
        assert np.array_equal(cnt, parts[0][2] + parts[1][2])
        assert ch == 15


def _fit_main(rank, world, port, X, C0, G, max_iter, tol, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        a, b = sharded.shard_rows(X.shape[0], world, rank)
        Xd = torch.from_numpy(np.ascontiguousarray(X[a:b])).cuda()
        r = sharded.fit_sharded(Xd, torch.from_numpy(C0).cuda(), G, max_iter, tol,
                                lambda t: dist.all_reduce(t, op=dist.ReduceOp.SUM))
        out.put((rank, a, r.labels.cpu().numpy(), r.centroids.cpu().numpy(), r.objective, r.n_iter,
                 [s["n_changed"] for s in r.stats]))
    finally:
        dist.destroy_process_group()


@pytest.mark.gpu
@pytest.mark.parametrize("G", [1, 26])
def test_sharded_fit_equals_single_fit(G):
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import oracle
    from paper_1905_09345_gb300 import build, kpynq, synth
    build.build()
    oracle.build()
    w = synth.anisotropic_1m(N=60001)
    X, C0 = w.X, w.C0
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_fit_main, args=(r, 2, port, X, C0, G, 30, 1e-4, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted([q.get(timeout=600) for _ in procs], key=lambda g: g[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    labels = np.concatenate([g[2] for g in got])
    C = got[0][3].astype(np.float64)
    assert np.array_equal(got[0][3], got[1][3]), "the shards' centroids differ"
    assert got[0][4] == got[1][4] and got[0][5] == got[1][5]
    # the oracle's FP64 argmin over the common centroids, and its J
    ref, _, _, _ = oracle.lloyd_assign(X.astype(np.float64), C)
    assert np.array_equal(labels, ref)
    J = oracle.lloyd_objective(X.astype(np.float64), labels, C)
    assert abs(got[0][4] - J) <= 1e-9 * J
    # the single-process fit
    km = kpynq.KMeans(torch.from_numpy(X).cuda(), torch.from_numpy(C0).cuda(), G)
    lab1 = torch.empty(X.shape[0], dtype=torch.int32, device="cuda")
    C1 = torch.empty(C0.shape, dtype=torch.float32, device="cuda")
    r = km.fit(30, 1e-4, lab1, C1)
    km.close()
    assert r.n_iter == got[0][5], (r.n_iter, got[0][5])
    assert [s["n_changed"] for s in r.stats] == got[0][6]
    C1 = C1.cpu().numpy().astype(np.float64)
    assert np.abs(C - C1).max() <= 1e-5 * max(1.0, np.abs(C1).max())
    assert np.array_equal(lab1.cpu().numpy(), labels)
