"""The multi-GPU bench path is N independent replicas (no collective on the
data path): each rank times its own steps, the job's time is the slowest
rank's, and the reported value is all ranks' units over that time.  Checked
here with two gloo ranks on the CPU."""
import os
import socket

import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(times[rank], dist, torch.device("cpu"))
        out.put((rank, t, bench.replica_value(world, 187_760_644, t)))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world, times = 2, [33.6e-6, 35.0e-6]
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, times, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in res:
        assert t == max(times)
        assert abs(v - 2 * 187_760_644 / max(times) / 1e9) < 1e-6


def test_single_rank_is_its_own_time():
    assert bench.max_over_ranks(1.5, None, None) == 1.5
    assert bench.replica_value(1, 2e9, 1.0) == 2.0
    assert bench.replica_value(4, 2e9, 1.0) == 8.0
