"""The bench's multi-rank bookkeeping on two gloo ranks (CPU): the job time is
the slowest rank's, the rate counts every rank's steps, each rank runs its own
sea (independent replicas, no data-path collective)."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    import bench
    from paper_2608_25203_b300 import seas
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.rank_env()
    ms = 100.0 + 50.0 * r                                   # rank 1 is slower
    job_ms = bench.max_over_ranks(ms, dist, device="cpu")
    eta, _, _ = seas.jonswap_sea(32, 32, 100.0, 100.0, 20.0, 1.0, 6.0, bench.replica_seed(r))
    q.put((r, w, local, job_ms, bench.job_rate(30, w, job_ms), float(eta[3, 5])))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[0] for x in res] == [0, 1] and all(x[1] == 2 and x[2] == x[0] for x in res)
    assert all(x[3] == 150.0 for x in res)                  # both ranks report the slowest rank's time
    assert all(abs(x[4] - 30 * 2 / 0.150) < 1e-9 for x in res)
    assert res[0][5] != res[1][5]                           # different seas per rank


def test_single_rank_defaults():
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.job_rate(10, 1, 100.0) == 100.0
    assert bench.replica_seed(0) == 3 and bench.replica_seed(5) == 8
    assert np.isfinite(bench.job_rate(1, 8, 1.0))
