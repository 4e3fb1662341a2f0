"""Sharding across ranks without a GPU: two gloo processes each compute their
block range (with the oracle standing in for the per-rank GPU step), the
query ciphertext is broadcast from rank 0 and the pieces are gathered back;
the result must equal the single-process run bit for bit."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1904_02033_b300.shard import distances_sharded, shard_blocks, shard_positions


def test_shard_blocks_cover_and_balance():
    for K in (1, 2, 3, 7, 123, 1221):
        for world in (1, 2, 3, 8):
            ranges = [shard_blocks(K, world, r) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == K
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1
    assert shard_positions(1000, 256, 3, 4) == (768, 1000)
    assert shard_positions(1000, 256, 4, 4) == (1000, 1000)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, result_q):
    from oracle.bfv import Oracle
    from paper_1904_02033_b300 import inputs

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        cfg = (256, 2, 40, 0, 5)
        n = 1000
        O = Oracle(*cfg)
        coords = inputs.uniform_coords(n, 5, 3)
        perm = inputs.permutation(n, 4)
        _, s_hat = O.keygen(5)
        q = inputs.uniform_coords(1, 5, 6)[0]
        ct_np = O.encrypt(s_hat, q, 7, 1) if rank == 0 else np.zeros((5, 2, 2, 256), np.uint64)
        ct = torch.from_numpy(ct_np.copy())

        def compute(ct_in, k0, k1):
            out, srv = O.distances(ct_in.numpy(), coords, perm, 8, 1, k0=k0, k1=k1)
            return torch.from_numpy(out), torch.from_numpy(srv)

        res = distances_sharded(compute, ct, n, 256, 2)
        if rank == 0:
            full_out, full_srv = O.distances(ct_np, coords, perm, 8, 1)
            result_q.put((np.array_equal(res[0].numpy(), full_out),
                          np.array_equal(res[1].numpy(), full_srv)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_run_equals_single_run(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert q.get(timeout=5) == (True, True)
