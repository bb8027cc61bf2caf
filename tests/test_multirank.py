"""The multi-rank benchmark path on CPU (gloo, world size 2): each rank runs
its own independent members (seed offset by rank), there is no collective on
the data path, and the reported time is the slowest rank's."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import torch.distributed as dist

    import bench
    from paper_2505_17025_gb300 import workloads as W
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        members = 3
        wl = W.slide_1d(n_members=members, nx=64, seed0=bench.rank_seed0(members, rank))
        ms = bench.max_over_ranks(10.0 + rank, ws, "cpu")
        amps = torch.tensor([m.A for m in wl.members], dtype=torch.float64)
        gathered = [torch.zeros_like(amps) for _ in range(ws)]
        dist.all_gather(gathered, amps)      # test only: compare the ranks' members
        out.put((rank, ms, [g.tolist() for g in gathered]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_weak_scaling_and_max_time():
    ctx = torch.multiprocessing.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = [out.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert [r[1] for r in res] == [11.0, 11.0]          # both ranks report the slowest
    a0, a1 = res[0][2]
    assert not np.allclose(a0, a1)                      # independent members per rank
    assert res[0][2] == res[1][2]
