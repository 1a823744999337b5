"""The N > 1 path of bench.py on the CPU: two `gloo` ranks, each with its own seeded batch
(weak scaling, no collective on the data path), the step time taken as the maximum over
ranks, and each rank's spot check against the oracle."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    import bench
    from oracle import plain
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        keys, idx, cts = bench.workload(rank)
        k = keys[idx[0]]
        m = plain.rsa_decrypt_crt(cts[0], k["p"], k["q"], k["dp"], k["dq"], k["qinv"])
        ok = plain.rsa_encrypt(m, k["e"], k["N"]) == cts[0]
        fake_ms = 10.0 + 5.0 * rank  # the slower rank decides the job's time
        slowest = bench.max_over_ranks(fake_ms, world, torch.device("cpu"))
        first = torch.tensor([cts[0] % (1 << 62)], dtype=torch.int64)
        gathered = [torch.zeros_like(first) for _ in range(world)]
        dist.all_gather(gathered, first)
        _, ridx, rops, rxs = bench.ragged_workload(rank, 64)
        out.put((rank, ok, slowest, [int(g.item()) for g in gathered], len(cts), rxs[0] % (1 << 62)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_own_batches_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    (r0, ok0, t0, g0, n0, x0), (r1, ok1, t1, g1, n1, x1) = res
    assert ok0 and ok1                      # each rank's spot check holds
    assert t0 == t1 == 15.0                 # both report the slowest rank's time
    assert g0 == g1 and g0[0] != g0[1]      # different, seeded batches per rank
    assert n0 == n1                         # the same work per rank (weak scaling)
    assert x0 != x1
