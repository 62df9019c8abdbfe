"""The multi-rank path of the benchmark on CPU: two processes over gloo
(127.0.0.1), each timing its own streams.  The job time is the slowest
rank's, the element count is every rank's work (weak scaling, no data
exchange between ranks), and each rank draws different inputs."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, ws, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank)})
    import bench
    import synth
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    w, r, local = bench._dist_env()
    assert (w, r, local) == (ws, rank, rank)
    # Rank-specific inputs (the bench seeds each rank's streams apart).
    x = synth.uniform(1000, seed=bench.SEEDS["uniform"] + 1000 * rank)
    elapsed, total, rate = bench.job_time(10.0 + 5.0 * rank, 12_000, ws)
    dist.barrier()
    q.put((rank, elapsed, total, rate, float(x[:10].sum())))
    dist.destroy_process_group()


def test_two_ranks_gloo():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, e0, t0, v0, s0), (r1, e1, t1, v1, s1) = out
    assert e0 == e1 == 15.0  # the slowest rank's time
    assert t0 == t1 == 24_000  # both ranks' elements
    assert v0 == pytest.approx(24_000 / 15e-3 / 1e9)
    assert s0 != s1  # different streams per rank


def test_single_rank_job_time():
    import bench
    assert bench.job_time(20.0, 1_000_000, 1) == (20.0, 1_000_000, 1_000_000 / 20e-3 / 1e9)
