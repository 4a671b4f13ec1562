"""The multi-rank path on CPU: slice blocks over ranks, and the rank-ordered exchange of
partial sums over gloo (world size 2 and 3) gives the full sliced amplitude of the oracle
(Eq. 2 across processes)."""

import os
import sys

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import socket

import pytest
import torch.multiprocessing as mp

from paper_2012_02430_gb300.dist import sharded_sum, slice_range


def test_slice_range_partitions():
    for n in (0, 1, 4, 7, 1024):
        for w in (1, 2, 3, 8):
            seen = []
            for r in range(w):
                lo, hi = slice_range(n, r, w)
                assert 0 <= lo <= hi <= n
                seen += list(range(lo, hi))
            assert seen == list(range(n))
    with pytest.raises(ValueError):
        slice_range(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from helpers import oracle_plan, oracle_problem
        from oracle import contract
        n, p, seed = 14, 3, 42
        edges, g, b, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
        plan = oracle_plan(adj, 0, 6, 3, 1)
        k = len(plan["sliced"])

        def partial(lo, count):
            tot, _ = contract.contract_amplitude(tensors, plan["order"], plan["sliced"],
                                                 plan["slice_step"], range(lo, lo + count))
            return tot * norm

        amp = sharded_sum(partial, 1 << k, rank, world)
        q.put((rank, amp, k))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_sum_over_gloo(world):
    import sys
    here = os.path.dirname(os.path.abspath(__file__))
    if here not in sys.path:
        sys.path.insert(0, here)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    results = [q.get(timeout=300) for _ in range(world)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    from helpers import oracle_plan, oracle_problem
    from oracle import contract
    edges, g, b, z, tensors, nv, norm, adj = oracle_problem(14, 3, 42)
    plan = oracle_plan(adj, 0, 6, 3, 1)
    assert len(plan["sliced"]) >= 2
    full, _ = contract.contract_amplitude(tensors, plan["order"], plan["sliced"], plan["slice_step"])
    amps = {r: a for r, a, _ in results}
    assert len(set(amps.values())) == 1  # identical on every rank (rank-ordered sum)
    assert abs(amps[0] - full * norm) <= 1e-12 * abs(full * norm)
