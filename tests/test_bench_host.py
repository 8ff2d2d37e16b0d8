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
    import argparse
    wl = bench.Normal32(argparse.Namespace(batch=2))
    a, b = wl.nets(0), wl.nets(1)
    for x in a:
        for y in b:
            assert not (x.data[0] == y.data[0]).all()


def test_ising_sweep_batches_hold_the_stored_betas_and_split_ranks():
    import argparse
    import numpy as np
    from tn_inputs import networks as nw
    wl = bench.Ising64(argparse.Namespace(batch=32))
    b0, b1 = wl.betas(0), wl.betas(1)
    assert len(b0) == len(b1) == 32 and len(set(b0)) == 32
    sweep = set(float(x) for x in nw.beta_sweep(256))
    assert set(b0) <= sweep and set(b1) <= sweep
    gold = [e["beta"] for e in wl.gold]
    assert b0[:len(gold)] == gold and b1[:len(gold)] == gold
    assert set(b0[len(gold):]).isdisjoint(b1[len(gold):])
    assert min(b0) == 0.2 and max(b0) == 0.7 and np.isclose(sorted(b0)[1] - sorted(b0)[0], 0.5 / 255 * 8, atol=0.1)


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
