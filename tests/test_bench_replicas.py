"""The replica path of bench.py (N > 1 processes, no data-path collective): every timed region is taken as the
slowest rank's and the whole-job rate sums the replicas.  Two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [3.0, 5.0][rank]
    ms = bench.max_over_ranks(local_ms, dist, "cpu")
    rate = bench.replica_rate(1000, ms / 1e3, world)
    out.put((rank, ms, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_replica_rate_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slower rank's time; the job processed 2 x 1000 units in 5 ms
    assert [r[1] for r in res] == [5.0, 5.0]
    assert all(abs(r[2] - 2000 / 5e-3) < 1e-6 for r in res)


def test_single_process_is_its_own_maximum():
    import bench
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.replica_rate(10, 2.0, 1) == 5.0
