"""Sharding across ranks without a GPU: gloo processes each compute their
share of the work (with the oracle standing in for the per-rank GPU step),
the query ciphertexts are broadcast from rank 0 and the pieces are gathered
back; the result must equal the single-process run bit for bit.  Covered:
the linear scan split by block ranges, with one and with several queries
per call, and the clustering gather split by query."""
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1904_02033_b300.shard import (assign_queries, distances_sharded, gather_sharded,
                                         shard_blocks, shard_positions)


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


def test_assign_queries_partitions_and_balances():
    rnd = np.random.default_rng(3)
    for world in (1, 2, 3, 8):
        for B in (0, 1, 5, 256):
            items = rnd.integers(1, 40, size=B)
            a = assign_queries(items, world)
            assert len(a) == world
            flat = sorted(b for part in a for b in part)
            assert flat == list(range(B))
            assert all(part == sorted(part) for part in a)
            if B >= world:
                loads = [int(items[part].sum()) if part else 0 for part in a]
                # longest-first: no rank exceeds the lightest by more than one query
                assert max(loads) - min(loads) <= int(items.max())
    assert assign_queries([5, 5, 5, 5], 2) == [[0, 2], [1, 3]]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


CFG = (256, 2, 40, 0, 5)


def _linear_scan_case(rank, B):
    """Oracle-side pieces of a small linear scan: B queries (ids 1, 4, 7, ..)
    over n = 1000 points, encrypted on rank 0 only."""
    from oracle.bfv import Oracle
    from paper_1904_02033_b300 import inputs

    n = 1000
    O = Oracle(*CFG)
    coords = inputs.uniform_coords(n, CFG[4], 3)
    perm = inputs.permutation(n, 4)
    _, s_hat = O.keygen(5)
    q = inputs.uniform_coords(B, CFG[4], 6)
    qids = [1 + 3 * b for b in range(B)]
    if rank == 0:
        ct_np = np.stack([O.encrypt(s_hat, q[b], 7, qids[b]) for b in range(B)])
    else:
        ct_np = np.zeros((B, CFG[4], 2, CFG[1], CFG[0]), np.uint64)
    return O, coords, perm, qids, n, ct_np


def _linear_worker(rank, world, port, B, result_q):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        O, coords, perm, qids, n, ct_np = _linear_scan_case(rank, B)
        ct = torch.from_numpy(ct_np.copy())

        def compute(ct_in, k0, k1):
            outs, srvs = [], []
            for b in range(B):
                o, s_ = O.distances(ct_in.numpy()[b], coords, perm, 8, qids[b], k0=k0, k1=k1)
                outs.append(o)
                srvs.append(s_)
            return torch.from_numpy(np.stack(outs)), torch.from_numpy(np.stack(srvs))

        res = distances_sharded(compute, ct, n, CFG[0], CFG[1])
        if rank == 0:
            ok = True
            for b in range(B):
                full_out, full_srv = O.distances(ct_np[b], coords, perm, 8, qids[b])
                ok &= np.array_equal(res[0].numpy()[b], full_out)
                ok &= np.array_equal(res[1].numpy()[b], full_srv)
            result_q.put((ok, tuple(res[0].shape), tuple(res[1].shape)))
    finally:
        dist.destroy_process_group()


def _gather_case():
    """Oracle-side pieces of a small clustering gather: n = 1500 points in 12
    clusters of skewed sizes (one empty), 5 queries probing 3 clusters each."""
    from paper_1904_02033_b300 import inputs

    n, C, B, P = 1500, 12, 5, 3
    rnd = np.random.default_rng(11)
    coords = inputs.uniform_coords(n, CFG[4], 12)
    assign = rnd.choice(C, size=n, p=inputs.zipf_weights(C, 1.1))
    assign[assign == C - 1] = 0
    offsets, members = inputs.clusters_csr(assign, C)
    probes = np.stack([rnd.permutation(C)[:P] for _ in range(B)]).astype(np.uint32)
    probes[1, 0] = C - 1
    lists = [np.concatenate([members[offsets[c]:offsets[c + 1]] for c in probes[b]]).astype(np.uint32)
             for b in range(B)]
    return coords, lists, [2 + b for b in range(B)]


def _gather_worker(rank, world, port, result_q):
    from oracle.bfv import Oracle
    from paper_1904_02033_b300 import inputs

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        O = Oracle(*CFG)
        coords, lists, qids = _gather_case()
        B = len(lists)
        _, s_hat = O.keygen(9)
        q = inputs.uniform_coords(B, CFG[4], 13)
        if rank == 0:
            ct_np = np.stack([O.encrypt(s_hat, q[b], 14, qids[b]) for b in range(B)])
        else:
            ct_np = np.zeros((B, CFG[4], 2, CFG[1], CFG[0]), np.uint64)
        blocks_b = [O.blocks(len(lst)) for lst in lists]
        points_b = [len(lst) for lst in lists]

        def one(ct_q, b):
            if len(lists[b]) == 0:
                return (np.zeros((0, 2, CFG[1], CFG[0]), np.uint64), np.zeros(0, np.uint32))
            return O.distances(ct_q, coords, lists[b], 15, qids[b])

        def compute(ct_sub, qs):
            res = [one(ct_sub.numpy()[i], b) for i, b in enumerate(qs)]
            return (torch.from_numpy(np.concatenate([r[0] for r in res])),
                    torch.from_numpy(np.concatenate([r[1] for r in res])),
                    torch.from_numpy(np.concatenate([lists[b] for b in qs])))

        res = gather_sharded(compute, torch.from_numpy(ct_np.copy()), blocks_b, points_b)
        if rank == 0:
            full = [one(ct_np[b], b) for b in range(B)]
            want_out = np.concatenate([f[0] for f in full])
            want_srv = np.concatenate([f[1] for f in full])
            want_ids = np.concatenate(lists)
            result_q.put((np.array_equal(res[0].numpy(), want_out),
                          np.array_equal(res[1].numpy(), want_srv),
                          np.array_equal(res[2].numpy(), want_ids)))
    finally:
        dist.destroy_process_group()


def _run(target, world, *args):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port) + args + (q,)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    return q.get(timeout=5)


@pytest.mark.parametrize("world,B", [(2, 1), (3, 1), (2, 3), (3, 4)])
def test_sharded_run_equals_single_run(world, B):
    ok, out_shape, srv_shape = _run(_linear_worker, world, B)
    assert ok
    assert out_shape == (B, 4, 2, CFG[1], CFG[0]) and srv_shape == (B, 1000)


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_gather_equals_single_run(world):
    assert _run(_gather_worker, world) == (True, True, True)
