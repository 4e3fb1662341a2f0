"""GPU parity of slot encoding (points in the CRT slots mod t): responses
bit-identical to the oracle's, server and client shares equal to the oracle's,
and the shares reconstruct the exact squared distances; on the per-query and
batched paths, with circuit privacy, through the allocating and the
allocation-free decryption."""
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


@pytest.mark.parametrize("cfg,n,B,batched,F", [
    ((256, 2, 40, 0, 5), 700, 2, False, 0),            # ragged last block
    ((64, 3, 50, 0, 3), 64 * 5, 3, False, 0),          # tiny N, full blocks
    ((8192, 3, 60, 0, 32), 20000, 1, False, 0),        # N = 8192, three 60-bit primes
    ((256, 2, 60, 0, 16), 256 * 9 + 3, 2, True, 0),    # tensor-core path
    ((8192, 3, 60, 0, 7), 8192 + 100, 1, False, 148),  # with circuit privacy
])
def test_slot_distances_match_oracle(cfg, n, B, batched, F):
    O = oracle(cfg)
    d = cfg[4]
    ctx = S.sanns_ctx_create(*cfg)
    S.sanns_set_encoding(ctx, True)
    coords = inputs.uniform_coords(n, d, n % 17)
    perm = inputs.permutation(n, 3)
    q = inputs.uniform_coords(B, d, 41)
    qids = np.arange(20, 20 + B, dtype=np.uint64)
    sk = S.sanns_keygen(ctx, 31)
    s, s_hat = O.keygen(31)
    db = S.sanns_encode_db(ctx, cu(coords), cu(perm))
    ct_in = S.sanns_encrypt_query(ctx, sk, cu(q), 32, cu(qids))
    pk = None
    if F:
        pk = S.sanns_public_key(ctx, sk, 33)
        S.sanns_set_circuit_privacy(ctx, pk, F)
        pk = pk.cpu().numpy()
    if batched:
        S.sanns_db_prepare_batched(ctx, db)
        out, srv = S.sanns_distances_batched(ctx, db, ct_in, 34, cu(qids))
        S.sanns_device_status(ctx)
    else:
        out, srv = S.sanns_distances(ctx, db, ct_in, 34, cu(qids))
    cli = S.sanns_decrypt_shares(ctx, sk, out, n, cu(q))
    cli_na = S.sanns_decrypt_shares_noalloc(ctx, sk, out, n, cu(q))
    torch.cuda.synchronize()
    out, srv, cli, cli_na = out.cpu().numpy(), srv.cpu().numpy(), cli.cpu().numpy(), cli_na.cpu().numpy()
    ct_np = ct_in.cpu().numpy()
    brute_all = coords[perm].astype(np.int64)
    for b in range(B):
        want_out, want_srv = O.distances(ct_np[b], coords, perm, 34, int(qids[b]), pk=pk,
                                         flood_bits=F, slots=True)
        assert np.array_equal(out[b], want_out), b
        assert np.array_equal(srv[b], want_srv), b
        want_cli = O.decrypt_shares(want_out, s, q[b], n, slots=True)
        assert np.array_equal(cli[b], want_cli), b
        assert np.array_equal(cli_na[b], want_cli), b
        brute = np.sum((brute_all - q[b].astype(np.int64)) ** 2, axis=1)
        assert np.array_equal((cli[b].astype(np.int64) + srv[b]) % O.t, brute), b


def test_slot_encoding_rejections():
    # t a power of two (t rule 1) has no 2N-th roots of unity
    ctx1 = S.sanns_ctx_create(256, 2, 40, 1, 4)
    with pytest.raises(S.SannsError):
        S.sanns_set_encoding(ctx1, True)
    ctx = S.sanns_ctx_create(256, 2, 40, 0, 4)
    coords = cu(inputs.uniform_coords(300, 4, 1))
    sk = S.sanns_keygen(ctx, 1)
    qids = cu(np.array([0], dtype=np.uint64))
    ct = S.sanns_encrypt_query(ctx, sk, cu(inputs.uniform_coords(1, 4, 2)), 3, qids)
    S.sanns_set_encoding(ctx, True)
    db_slots = S.sanns_encode_db(ctx, coords)
    S.sanns_set_encoding(ctx, False)
    with pytest.raises(S.SannsError):          # the database's encoding differs
        S.sanns_distances(ctx, db_slots, ct, 4, qids)
    S.sanns_set_encoding(ctx, True)
    S.sanns_distances(ctx, db_slots, ct, 4, qids)   # the matching setting works


@pytest.mark.parametrize("cfg,n,F", [((256, 2, 40, 0, 5), 700, 0), ((8192, 3, 60, 0, 7), 8192 + 100, 148)])
def test_slot_encoding_with_ntt_form_responses(cfg, n, F):
    # the NTT-form response is the NTT of the slot-encoded coefficient
    # response, and NTT-form decryption decodes the slots
    O = oracle(cfg)
    d = cfg[4]
    ctx = S.sanns_ctx_create(*cfg)
    S.sanns_set_encoding(ctx, True)
    S.sanns_set_response_form(ctx, True)
    coords = inputs.uniform_coords(n, d, 21)
    perm = inputs.permutation(n, 22)
    q = inputs.uniform_coords(1, d, 23)
    qids = np.array([9], dtype=np.uint64)
    sk = S.sanns_keygen(ctx, 24)
    s, s_hat = O.keygen(24)
    db = S.sanns_encode_db(ctx, cu(coords), cu(perm))
    ct_in = S.sanns_encrypt_query(ctx, sk, cu(q), 25, cu(qids))
    pk = None
    if F:
        pk_d = S.sanns_public_key(ctx, sk, 26)
        S.sanns_set_circuit_privacy(ctx, pk_d, F)
        pk = pk_d.cpu().numpy()
    out, srv = S.sanns_distances(ctx, db, ct_in, 27, cu(qids))
    cli = S.sanns_decrypt_shares(ctx, sk, out, n, cu(q)).cpu().numpy()[0]
    want_out, want_srv = O.distances(ct_in.cpu().numpy()[0], coords, perm, 27, 9, pk=pk, flood_bits=F,
                                     slots=True)
    assert np.array_equal(out.cpu().numpy()[0], O.to_ntt_form(want_out))
    assert np.array_equal(srv.cpu().numpy()[0], want_srv)
    assert np.array_equal(cli, O.decrypt_shares(want_out, s, q[0], n, slots=True))
    brute = np.sum((coords[perm].astype(np.int64) - q[0].astype(np.int64)) ** 2, axis=1)
    assert np.array_equal((cli.astype(np.int64) + srv.cpu().numpy()[0]) % O.t, brute)
