"""GPU parity of circuit privacy (public-key re-randomisation plus noise
flooding): every ciphertext bit-identical to the oracle's, and the shares
still reconstruct the exact squared distances."""
import numpy as np
import pytest
import torch

from oracle.bfv import Oracle
from paper_1904_02033_b300 import inputs
from paper_1904_02033_b300 import sanns as S

pytestmark = pytest.mark.gpu

_O = {}


def oracle(cfg):
    if cfg not in _O:
        _O[cfg] = Oracle(*cfg)
    return _O[cfg]


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("cfg", [(256, 2, 60, 0, 5), (8192, 3, 60, 0, 7)])
def test_public_key_matches_oracle(cfg):
    ctx = S.sanns_ctx_create(*cfg)
    sk = S.sanns_keygen(ctx, 51)
    pk = S.sanns_public_key(ctx, sk, 52)
    O = oracle(cfg)
    _, s_hat = O.keygen(51)
    assert np.array_equal(pk.cpu().numpy(), O.public_key(s_hat, 52))
    assert S.sanns_circuit_privacy_max_flood_bits(ctx) == O.max_flood_bits()


@pytest.mark.parametrize("cfg,n,B,F,batched", [
    ((256, 3, 60, 0, 5), 256 * 3 - 7, 2, 100, False),
    ((8192, 3, 60, 0, 7), 8192 * 2 - 100, 1, 148, False),   # 108 bits over ~2^40 of noise
    ((256, 2, 60, 0, 16), 256 * 9 + 3, 3, 60, True),
])
def test_private_distances_match_oracle(cfg, n, B, F, batched):
    O = oracle(cfg)
    ctx = S.sanns_ctx_create(*cfg)
    d = cfg[4]
    coords = inputs.uniform_coords(n, d, n % 13)
    perm = inputs.permutation(n, 5)
    q = inputs.uniform_coords(B, d, 77)
    qids = np.arange(60, 60 + B, dtype=np.uint64)
    sk = S.sanns_keygen(ctx, 61)
    pk = S.sanns_public_key(ctx, sk, 62)
    db = S.sanns_encode_db(ctx, cu(coords), cu(perm))
    ct_in = S.sanns_encrypt_query(ctx, sk, cu(q), 63, cu(qids))
    plain_out, _ = S.sanns_distances(ctx, db, ct_in, 64, cu(qids))
    S.sanns_set_circuit_privacy(ctx, pk, F)
    if batched:
        S.sanns_db_prepare_batched(ctx, db)
        out, srv = S.sanns_distances_batched(ctx, db, ct_in, 64, cu(qids))
        S.sanns_device_status(ctx)
        pq_out, pq_srv = S.sanns_distances(ctx, db, ct_in, 64, cu(qids))
        assert torch.equal(out, pq_out) and torch.equal(srv, pq_srv)
    else:
        out, srv = S.sanns_distances(ctx, db, ct_in, 64, cu(qids))
    out, srv = out.cpu().numpy(), srv.cpu().numpy()
    s, s_hat = O.keygen(61)
    opk = O.public_key(s_hat, 62)
    cti = ct_in.cpu().numpy()
    for b in range(B if cfg[0] <= 256 else 1):
        oo, os_ = O.distances(cti[b], coords, perm, 64, int(qids[b]), pk=opk, flood_bits=F)
        assert np.array_equal(out[b], oo)
        assert np.array_equal(srv[b], os_)
    for b in range(B):
        cli = O.decrypt_shares(out[b], s, q[b], n)
        brute = np.sum((coords[perm].astype(np.int64) - q[b].astype(np.int64)) ** 2, axis=1)
        assert np.array_equal((cli.astype(np.int64) + srv[b]) % O.t, brute)
    # off again: the plain responses come back
    S.sanns_set_circuit_privacy(ctx, None)
    again, _ = S.sanns_distances(ctx, db, ct_in, 64, cu(qids))
    assert torch.equal(again, plain_out)


def test_flood_bits_bound():
    cfg = (256, 2, 40, 0, 4)
    ctx = S.sanns_ctx_create(*cfg)
    sk = S.sanns_keygen(ctx, 1)
    pk = S.sanns_public_key(ctx, sk, 2)
    fmax = S.sanns_circuit_privacy_max_flood_bits(ctx)
    assert fmax == oracle(cfg).max_flood_bits()
    with pytest.raises(S.SannsError) as e:
        S.sanns_set_circuit_privacy(ctx, pk, fmax + 1)
    assert e.value.code == -1
    S.sanns_set_circuit_privacy(ctx, pk, fmax)


@pytest.mark.parametrize("cfg", [(256, 2, 40, 0, 4), (256, 3, 60, 0, 8)])
def test_maximum_flooding_extreme_coordinates(cfg):
    # the largest allowed flooding exponent with the extreme coordinates (0
    # against 255): bit-identical to the oracle, and the GPU decryption still
    # reconstructs every distance
    O = oracle(cfg)
    ctx = S.sanns_ctx_create(*cfg)
    N, d = cfg[0], cfg[4]
    n = 2 * N - 3
    coords = np.full((n, d), 255, dtype=np.uint8)
    coords[1::3] = 0
    q = np.stack([np.zeros(d, dtype=np.uint8), np.full(d, 255, dtype=np.uint8)])
    qids = np.array([9, 10], dtype=np.uint64)
    sk = S.sanns_keygen(ctx, 81)
    pk = S.sanns_public_key(ctx, sk, 82)
    F = S.sanns_circuit_privacy_max_flood_bits(ctx)
    S.sanns_set_circuit_privacy(ctx, pk, F)
    db = S.sanns_encode_db(ctx, cu(coords))
    ct_in = S.sanns_encrypt_query(ctx, sk, cu(q), 83, cu(qids))
    out, srv = S.sanns_distances(ctx, db, ct_in, 84, cu(qids))
    cli = S.sanns_decrypt_shares(ctx, sk, out, n, cu(q)).cpu().numpy()
    out, srv = out.cpu().numpy(), srv.cpu().numpy()
    s, s_hat = O.keygen(81)
    opk = O.public_key(s_hat, 82)
    cti = ct_in.cpu().numpy()
    for b in range(2):
        oo, os_ = O.distances(cti[b], coords, None, 84, int(qids[b]), pk=opk, flood_bits=F)
        assert np.array_equal(out[b], oo) and np.array_equal(srv[b], os_)
        brute = np.sum((coords.astype(np.int64) - q[b].astype(np.int64)) ** 2, axis=1)
        assert np.array_equal((cli[b].astype(np.int64) + srv[b]) % O.t, brute)
