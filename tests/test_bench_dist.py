"""bench.py's multi-rank timing plumbing on CPU: two gloo ranks.

Under torchrun every rank runs its own replica problem (no collective on the
data path); the step time reported is the maximum over ranks and the units
are summed over ranks.  This runs bench.aggregate and bench.barrier in two
spawned processes with the gloo backend and checks both reductions.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        ms, units = bench.aggregate(10.0 + 5.0 * rank, 1000.0 * (rank + 1), world)
        bench.barrier(world)
        out.put((rank, ms, units, bench.dist_env()))
    finally:
        dist.destroy_process_group()


def test_aggregate_max_time_sum_units_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, units, env in res:
        assert ms == 15.0            # max over ranks
        assert units == 3000.0       # sum over ranks
        assert env == (2, rank, 0)   # WORLD_SIZE, RANK, LOCAL_RANK (unset -> 0)


def test_aggregate_single_rank_is_identity():
    import bench
    assert bench.aggregate(7.5, 42.0, 1) == (7.5, 42.0)


def test_energy_per_point_iteration():
    import bench
    e = bench.energy_of(3.0e9, {"power_w_mean": 600.0, "samples": 7})
    assert e["value"] == 3.0e9 / 600.0 and e["unit"] == "points*iters/J"
    assert bench.energy_of(1.0, {"power_w_mean": None}) is None
