"""Host-side logic of bench.py on CPU: clock parsing, per-rank sharding, max over ranks (gloo)."""
import os
import socket

import pytest

import bench


def test_parse_clocks(tmp_path):
    p = tmp_path / "c.csv"
    p.write_text("0, 1900, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Active\n"
                 "0, 1950, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                 "0, 2000, 2070, 980.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    s = bench.parse_clocks(str(p))
    assert s["sm_mhz"] == 1950 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3
    assert bench.parse_clocks(str(tmp_path / "missing.csv")) is None


def test_ranks_get_disjoint_seeds():
    a, _ = bench.build_inputs(0, 2)
    b, _ = bench.build_inputs(1, 2)
    for x in a:
        for y in b:
            assert not (x.data[0] == y.data[0]).all()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dev = torch.device("cpu")
    bench.barrier(dev)
    m = bench.max_over_ranks(10.0 * (rank + 1), dev)
    q.put((rank, m))
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert out == [(0, 20.0), (1, 20.0)]
