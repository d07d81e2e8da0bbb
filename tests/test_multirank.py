"""Multi-rank host logic on CPU with gloo (world size 2): plume sharding covers every plume once
and balances the estimated cost; the whole-job throughput is sum(units) / max(time) on every
rank; single-plume replicas each report their own work."""
import os
import socket

import pytest

from paper_2108_09488_gb300 import inputs, sharding


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    plumes = inputs.batched_2d()
    costs = [sharding.plume_cost(p) for p in plumes]
    shards = sharding.shard_plumes(costs, world)
    mine = shards[rank]
    units = sum(2.0 * costs[i] for i in mine)
    ms = 10.0 + rank           # a slower second rank
    value, max_ms, total = sharding.aggregate(units, ms)
    q.put((rank, mine, units, value, max_ms, total))
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_two_ranks_shard_and_aggregate():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, u0, v0, m0, t0), (r1, s1, u1, v1, m1, t1) = res
    assert sorted(s0 + s1) == list(range(64)) and not set(s0) & set(s1)
    assert abs(u0 - u1) / (u0 + u1) < 0.02            # LPT balance of the estimated cost
    assert m0 == m1 == 11.0 and t0 == t1 == pytest.approx(u0 + u1)
    assert v0 == v1 == pytest.approx((u0 + u1) / 11.0e-3)


def test_shard_plumes_deterministic_and_single_rank():
    costs = [5.0, 1.0, 3.0, 3.0, 2.0]
    assert sharding.shard_plumes(costs, 1) == [[0, 1, 2, 3, 4]]
    a = sharding.shard_plumes(costs, 3)
    assert a == sharding.shard_plumes(costs, 3)
    assert sorted(sum(a, [])) == list(range(5))
    value, ms, units = sharding.aggregate(100.0, 2.0)
    assert value == 100.0 / 2e-3 and ms == 2.0 and units == 100.0
