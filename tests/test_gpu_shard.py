"""Shard databases on one GPU (the per-rank compute step of the multi-GPU
split): block-range shards encoded from slices of the permuted list with
their position base reproduce the single-database run bit for bit."""
import numpy as np
import pytest
import torch

from paper_1904_02033_b300 import inputs
from paper_1904_02033_b300 import sanns as S
from paper_1904_02033_b300.shard import gpu_shard_compute, shard_blocks

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("world", [2, 3])
def test_gpu_shards_concatenate_to_full_run(world):
    ctx = S.sanns_ctx_create(4096, 2, 54, 0, 16)
    n = 4096 * 5 - 123
    coords = torch.from_numpy(inputs.uniform_coords(n, 16, 1)).cuda()
    perm = torch.from_numpy(inputs.permutation(n, 2)).cuda()
    sk = S.sanns_keygen(ctx, 3)
    q = torch.from_numpy(inputs.uniform_coords(1, 16, 4)).cuda()
    qids = torch.tensor([9], dtype=torch.int64).to(torch.uint64).cuda()
    ct = S.sanns_encrypt_query(ctx, sk, q, 5, qids)
    full = S.sanns_encode_db(ctx, coords, perm)
    out, srv = S.sanns_distances(ctx, full, ct, 6, qids)
    compute = gpu_shard_compute(ctx, coords, perm, n, 6, qids)
    K = full.K
    outs, srvs = [], []
    for r in range(world):
        k0, k1 = shard_blocks(K, world, r)
        o, s_ = compute(ct, k0, k1)
        outs.append(o)
        srvs.append(s_)
    torch.cuda.synchronize()
    assert torch.equal(torch.cat(outs).cpu(), out[0].cpu())
    assert torch.equal(torch.cat(srvs).cpu(), srv[0].cpu())
