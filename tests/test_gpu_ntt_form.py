"""NTT-form responses: bit for bit the NTT of the coefficient-form responses
(oracle), decrypted by the client to the same shares, on the per-query and
batched paths, with and without circuit privacy."""
import numpy as np
import pytest
import torch

from oracle.bfv import Oracle
from paper_1904_02033_b300 import inputs
from paper_1904_02033_b300 import sanns as S

pytestmark = pytest.mark.gpu


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("cfg,n,B,privacy,batched", [
    ((256, 2, 60, 0, 6), 256 * 4 - 9, 2, False, False),
    ((8192, 3, 60, 0, 8), 8192 * 2 - 33, 1, False, False),
    ((256, 3, 60, 0, 5), 256 * 3 + 1, 2, True, False),
    ((256, 2, 60, 0, 16), 256 * 9 - 1, 3, False, True),
    ((256, 2, 60, 0, 16), 256 * 5 + 7, 3, True, True),
    # every count of leading radix-2 stages of the fused mask transform
    # (log2 N mod 4 = 0, 1, 2, 3), ragged last blocks
    ((4096, 2, 54, 0, 8), 4096 * 2 - 5, 2, False, False),
    ((64, 2, 50, 0, 3), 64 * 5 - 3, 2, False, False),
    ((16384, 2, 60, 0, 4), 16384 + 77, 1, False, False),
    ((2048, 2, 50, 0, 4), 2048 * 3 - 1, 2, False, True),
])
def test_ntt_form_responses(cfg, n, B, privacy, batched):
    O = Oracle(*cfg)
    ctx = S.sanns_ctx_create(*cfg)
    d = cfg[4]
    coords = inputs.uniform_coords(n, d, 3)
    perm = inputs.permutation(n, 4)
    q = inputs.uniform_coords(B, d, 5)
    qids = cu(np.arange(7, 7 + B, dtype=np.uint64))
    sk = S.sanns_keygen(ctx, 8)
    db = S.sanns_encode_db(ctx, cu(coords), cu(perm))
    ct = S.sanns_encrypt_query(ctx, sk, cu(q), 9, qids)
    F = 60
    if privacy:
        pk = S.sanns_public_key(ctx, sk, 10)
        S.sanns_set_circuit_privacy(ctx, pk, F)
    coef, srv_c = S.sanns_distances(ctx, db, ct, 11, qids)
    S.sanns_set_response_form(ctx, True)
    if batched:
        S.sanns_db_prepare_batched(ctx, db)
        out, srv = S.sanns_distances_batched(ctx, db, ct, 11, qids)
        S.sanns_device_status(ctx)
    else:
        out, srv = S.sanns_distances(ctx, db, ct, 11, qids)
    assert torch.equal(srv, srv_c)
    coef_np, out_np = coef.cpu().numpy(), out.cpu().numpy()
    s, s_hat = O.keygen(8)
    for b in range(min(B, 2)):
        assert np.array_equal(out_np[b], O.to_ntt_form(coef_np[b]))
    if cfg[0] <= 256:
        opk = O.public_key(s_hat, 10) if privacy else None
        oo, _ = O.distances(ct.cpu().numpy()[0], coords, perm, 11, 7, pk=opk, flood_bits=F)
        assert np.array_equal(out_np[0], O.to_ntt_form(oo))
    cli = S.sanns_decrypt_shares(ctx, sk, out, n, cu(q))
    S.sanns_set_response_form(ctx, False)
    cli_c = S.sanns_decrypt_shares(ctx, sk, coef, n, cu(q))
    assert torch.equal(cli, cli_c)
    brute = np.sum((coords[perm].astype(np.int64)[None] - q.astype(np.int64)[:, None]) ** 2, axis=2)
    assert np.array_equal((cli.cpu().numpy().astype(np.int64) + srv.cpu().numpy()) % O.t, brute)
