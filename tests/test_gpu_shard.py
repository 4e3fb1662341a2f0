"""Shards on one GPU (the per-rank compute steps of the multi-GPU split, run
one after another): block-range shard databases encoded from slices of the
permuted list with their position base reproduce the single-database run
bit for bit, for several queries per call on the per-query and on the
tensor-core path; and the clustering gather split by query (each rank's
queries in one call) reassembles to the single call."""
import numpy as np
import pytest
import torch

from paper_1904_02033_b300 import inputs
from paper_1904_02033_b300 import sanns as S
from paper_1904_02033_b300.shard import (assign_queries, gpu_gather_compute, gpu_shard_compute,
                                         shard_blocks)

pytestmark = pytest.mark.gpu


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("world,B,batched", [(2, 1, False), (3, 1, False), (3, 5, False),
                                             (2, 6, True), (4, 3, True)])
def test_gpu_shards_concatenate_to_full_run(world, B, batched):
    ctx = S.sanns_ctx_create(4096, 2, 54, 0, 16)
    n = 4096 * 9 - 123
    coords = cu(inputs.uniform_coords(n, 16, 1))
    perm = cu(inputs.permutation(n, 2))
    sk = S.sanns_keygen(ctx, 3)
    q = cu(inputs.uniform_coords(B, 16, 4))
    qids = cu(np.arange(9, 9 + B, dtype=np.uint64))
    ct = S.sanns_encrypt_query(ctx, sk, q, 5, qids)
    full = S.sanns_encode_db(ctx, coords, perm)
    out, srv = S.sanns_distances(ctx, full, ct, 6, qids)
    compute = gpu_shard_compute(ctx, coords, perm, n, 6, qids, batched=batched)
    K = full.K
    outs, srvs = [], []
    for r in range(world):
        k0, k1 = shard_blocks(K, world, r)
        o, s_ = compute(ct, k0, k1)
        assert o.shape == (B, k1 - k0, 2, ctx.L, ctx.N)
        outs.append(o.cpu())
        srvs.append(s_.cpu())
    S.sanns_device_status(ctx)
    assert torch.equal(torch.cat([o.view(torch.int64) for o in outs], 1).view(torch.uint64), out.cpu())
    assert torch.equal(torch.cat([s_.view(torch.int32) for s_ in srvs], 1).view(torch.uint32), srv.cpu())


@pytest.mark.parametrize("world", [2, 3])
def test_gpu_gather_split_by_query_reassembles(world):
    cfg = (256, 2, 40, 0, 5)
    n, C, B, P = 3000, 20, 7, 4
    rnd = np.random.default_rng(5)
    coords = inputs.uniform_coords(n, cfg[4], 1)
    assign = rnd.choice(C, size=n, p=inputs.zipf_weights(C, 1.1))
    offsets, members = inputs.clusters_csr(assign, C)
    probes = np.stack([rnd.permutation(C)[:P] for _ in range(B)]).astype(np.uint32)
    ctx = S.sanns_ctx_create(*cfg)
    sk = S.sanns_keygen(ctx, 3)
    cl = S.sanns_clusters_create(ctx, cu(coords), offsets, cu(members))
    qids = cu(np.arange(30, 30 + B, dtype=np.uint64))
    ct = S.sanns_encrypt_query(ctx, sk, cu(inputs.uniform_coords(B, cfg[4], 2)), 4, qids)
    ref_out, ref_srv, ref_ids, n_b, k_b = S.sanns_distances_gather(ctx, cl, ct, probes, 6, qids)
    compute = gpu_gather_compute(ctx, cl, probes, 6, qids)
    parts = {}
    for qs in assign_queries(k_b, world):
        if not qs:
            continue
        idx = torch.as_tensor(qs, dtype=torch.int64, device="cuda")
        o, s_, i_ = compute(ct.view(torch.int64)[idx].contiguous().view(torch.uint64), qs)
        ko = no = 0
        for b in qs:
            parts[b] = (o[ko:ko + int(k_b[b])].cpu(), s_[no:no + int(n_b[b])].cpu(), i_[no:no + int(n_b[b])].cpu())
            ko += int(k_b[b])
            no += int(n_b[b])
    cat = lambda k, dt, st: torch.cat([parts[b][k].view(st) for b in range(B)]).view(dt)
    assert torch.equal(cat(0, torch.uint64, torch.int64), ref_out.cpu())
    assert torch.equal(cat(1, torch.uint32, torch.int32), ref_srv.cpu())
    assert torch.equal(cat(2, torch.uint32, torch.int32), ref_ids.cpu())
