"""Failure detection without faulting the GPU: a bounded device-side wait
that must time out reports SANNS_ETIMEOUT through the host and leaves the
context usable; a corrupted response coefficient is caught by the share
reconstruction at exactly the corrupted position."""
import numpy as np
import pytest
import torch

from paper_1904_02033_b300 import inputs
from paper_1904_02033_b300 import sanns as S

pytestmark = pytest.mark.gpu


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _distances(ctx, n, d, seed):
    coords = inputs.uniform_coords(n, d, seed)
    q = inputs.uniform_coords(1, d, seed + 1)
    qids = cu(np.array([seed], dtype=np.uint64))
    sk = S.sanns_keygen(ctx, seed)
    db = S.sanns_encode_db(ctx, cu(coords))
    ct = S.sanns_encrypt_query(ctx, sk, cu(q), seed + 2, qids)
    out, srv = S.sanns_distances(ctx, db, ct, seed + 3, qids)
    brute = np.sum((coords.astype(np.int64) - q[0].astype(np.int64)) ** 2, axis=1)
    return sk, q, out, srv, brute


def test_bounded_wait_times_out_and_context_stays_usable():
    ctx = S.sanns_ctx_create(256, 2, 40, 0, 5)
    S.sanns_device_status(ctx)                       # clean to start with
    S.sanns_selftest_wait_timeout(ctx, 20)
    with pytest.raises(S.SannsError) as e:
        S.sanns_device_status(ctx)
    assert e.value.code == -4                        # SANNS_ETIMEOUT
    S.sanns_device_status(ctx)                       # read once, then cleared
    for bad in (0, 1001):
        with pytest.raises(S.SannsError):
            S.sanns_selftest_wait_timeout(ctx, bad)
    # the same context still computes exact distances
    sk, q, out, srv, brute = _distances(ctx, 600, 5, 7)
    cli = S.sanns_decrypt_shares(ctx, sk, out, 600, cu(q))
    t = ctx.query()["t"]
    assert np.array_equal((cli.cpu().numpy()[0].astype(np.int64) + srv.cpu().numpy()[0]) % t, brute)
    S.sanns_device_status(ctx)


def test_corrupted_response_is_detected_at_its_position():
    ctx = S.sanns_ctx_create(256, 2, 40, 0, 5)
    n = 600
    sk, q, out, srv, brute = _distances(ctx, n, 5, 11)
    t = ctx.query()["t"]
    x = 137
    bad_h = out.cpu().numpy().copy()
    bad_h[0, 0, 0, 0, x] ^= np.uint64(1 << 30)          # c0, prime 0, coefficient x
    bad = cu(bad_h)
    ok_rec = (S.sanns_decrypt_shares(ctx, sk, out, n, cu(q)).cpu().numpy()[0].astype(np.int64)
              + srv.cpu().numpy()[0]) % t
    bad_rec = (S.sanns_decrypt_shares(ctx, sk, bad, n, cu(q)).cpu().numpy()[0].astype(np.int64)
               + srv.cpu().numpy()[0]) % t
    assert np.array_equal(ok_rec, brute)
    assert np.flatnonzero(bad_rec != brute).tolist() == [x]
