"""The batch partitioner on two CPU ranks (gloo): every problem lands on
exactly one rank, both ranks compute the same assignment independently, and
the modelled loads are balanced within the largest single problem."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import __graft_entry__ as g  # noqa: F401  (sys.path)
    from paper_0707_2347_gb300 import partition
    shapes = synth.batch_shapes(64, 384, 6144)
    parts, cost = partition.assign(shapes, world)
    mine = torch.tensor(parts[rank] + [-1] * (len(shapes) - len(parts[rank])))
    gathered = [torch.zeros_like(mine) for _ in range(world)]
    dist.all_gather(gathered, mine)
    loads = torch.tensor([sum(cost[i] for i in parts[r]) for r in range(world)], dtype=torch.float64)
    loads_all = [torch.zeros_like(loads) for _ in range(world)]
    dist.all_gather(loads_all, loads)
    if rank == 0:
        got = sorted(int(x) for t in gathered for x in t.tolist() if x >= 0)
        same = all(torch.equal(loads_all[0], l) for l in loads_all)
        q.put((got, len(shapes), loads.tolist(), max(cost), same))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_partition_covers_and_balances():
    pytest.importorskip("torch.distributed")
    import __graft_entry__ as g
    g.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got, total, loads, biggest, same = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert got == list(range(total))
    assert same
    assert abs(loads[0] - loads[1]) <= biggest + 1e-6
