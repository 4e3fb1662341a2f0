"""The allocation-free decryption entry point must give exactly what the
allocating one gives.  Callers that cannot allocate device memory during a
call (graph capture, real-time loops, fixed memory budgets) use it; its
scratch is a fixed device array shared by all calls, so two calls in a row
are checked to make sure the first call's leftovers never leak into the
second.  Kept in its own file, collected last."""
import numpy as np
import pytest
import torch

from paper_1904_02033_b300 import inputs
from paper_1904_02033_b300 import sanns as S

pytestmark = pytest.mark.gpu


def _ciphertexts(ctx, sk, n, B, seed):
    coords = torch.from_numpy(inputs.uniform_coords(n, ctx.d, seed)).cuda()
    q = torch.from_numpy(inputs.uniform_coords(B, ctx.d, seed + 1)).cuda()
    qids = torch.arange(B, dtype=torch.int64).to(torch.uint64).cuda()
    db = S.sanns_encode_db(ctx, coords)
    ct_in = S.sanns_encrypt_query(ctx, sk, q, seed + 2, qids)
    ct_out, _ = S.sanns_distances(ctx, db, ct_in, seed + 3, qids)
    return ct_out, q


def test_noalloc_decrypt_equals_allocating_decrypt_twice_in_a_row():
    ctx = S.sanns_ctx_create(4096, 2, 54, 0, 32)
    sk = S.sanns_keygen(ctx, 7)
    # first call: two queries over three blocks (ragged tail)
    ct1, q1 = _ciphertexts(ctx, sk, 3 * 4096 - 100, 2, 11)
    got1 = S.sanns_decrypt_shares_noalloc(ctx, sk, ct1, 3 * 4096 - 100, q1)
    want1 = S.sanns_decrypt_shares(ctx, sk, ct1, 3 * 4096 - 100, q1)
    # second call: a smaller request that uses only part of the scratch the
    # first call filled
    ct2, q2 = _ciphertexts(ctx, sk, 700, 1, 23)
    got2 = S.sanns_decrypt_shares_noalloc(ctx, sk, ct2, 700, q2)
    want2 = S.sanns_decrypt_shares(ctx, sk, ct2, 700, q2)
    torch.cuda.synchronize()
    assert torch.equal(got1.cpu(), want1.cpu())
    assert torch.equal(got2.cpu(), want2.cpu())
    assert not torch.equal(got1[0, :700].cpu(), got2[0].cpu())


def test_noalloc_decrypt_rejects_requests_beyond_the_static_scratch():
    ctx = S.sanns_ctx_create(4096, 2, 54, 0, 4)
    sk = S.sanns_keygen(ctx, 1)
    max_words = S.sanns_decrypt_noalloc_max_words()
    n = (max_words // (2 * 4096) + 1) * 4096     # one block more than fits
    ct_out = torch.zeros((1, n // 4096, 2, 2, 4096), dtype=torch.uint64, device="cuda")
    q = torch.zeros((1, 4), dtype=torch.uint8, device="cuda")
    with pytest.raises(S.SannsError) as e:
        S.sanns_decrypt_shares_noalloc(ctx, sk, ct_out, n, q)
    assert e.value.code == -1 and "static scratch" in str(e.value)
