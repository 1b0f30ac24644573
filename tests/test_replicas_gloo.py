"""The multi-GPU path is replicas (the solve needs no exchange): each rank
solves its own copy of the family (its own order of the sequences), and the
bench reports the slowest rank's time over all the solves of the job.
Checked here with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [1.0, 3.0][rank]  # rank 1 is the slow one
        v = bench.job_seconds_per_solve(local, steps=4, world=world, dist=dist)
        import numpy as np
        msa = np.arange(40, dtype=np.int8).reshape(10, 4) % 21
        q.put((rank, v, bench.replica_msa(msa, rank).tobytes()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_and_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = dict((r, (v, s)) for r, v, s in (q.get(timeout=5) for _ in range(2)))
    # max over ranks (3.0 s) over 4 steps x 2 ranks
    assert got[0][0] == pytest.approx(3.0 / 8) and got[1][0] == pytest.approx(3.0 / 8)
    # each rank its own copy: rank 0 the data as generated, rank 1 the same
    # rows in another order
    import numpy as np
    msa = np.arange(40, dtype=np.int8).reshape(10, 4) % 21
    r0 = np.frombuffer(got[0][1], np.int8).reshape(10, 4)
    r1 = np.frombuffer(got[1][1], np.int8).reshape(10, 4)
    assert np.array_equal(r0, msa) and not np.array_equal(r1, msa)
    assert sorted(map(bytes, r1)) == sorted(map(bytes, msa))


def test_single_rank_value():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_seconds_per_solve(2.5, steps=5, world=1) == pytest.approx(0.5)
