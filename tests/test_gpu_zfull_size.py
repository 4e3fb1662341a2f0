"""Parity at the full sizes the benchmark times.

Linear scan: n = 10^6 points of a 64-component Gaussian mixture, d = 128,
N = 8192, three 60-bit primes, one query, every MAC launch variant (the
autotuned one first, as the benchmark runs it).

Batched (tensor-core) path: n = 10^7 points of a 256-component mixture
(sigma 12), d = 96, 64 queries in one call, in the tile shape the autotuner
picks, as the benchmark runs it.

The oracle computes sampled blocks one by one (the first, a middle one and
the ragged last, with their server and client shares); every position's
shares reconstruct the brute-force squared distance.  The file sorts after
the other GPU tests, so the small cases report first."""
import numpy as np
import pytest
import torch

from oracle.bfv import Oracle
from paper_1904_02033_b300 import inputs
from paper_1904_02033_b300 import sanns as S

pytestmark = pytest.mark.gpu

CFG = (8192, 3, 60, 0, 128)
N_POINTS = 1_000_000


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _inputs(n, d):
    coords = inputs.mixture_coords(n, d, 64, 20.0, 2, means_seed=1)
    perm = inputs.permutation(n, 3)
    q = inputs.mixture_coords(1, d, 64, 20.0, 4, means_seed=1)
    return coords, perm, q


def _gpu_run(cfg, coords, perm, q, qid, key_seed, enc_seed, mask_seed):
    """The library's outputs: the query ciphertext, then per MAC variant the
    responses and server shares, and the client shares (numpy)."""
    N, L, _, _, _ = cfg
    n = len(perm)
    K = -(-n // N)
    ctx = S.sanns_ctx_create(*cfg)
    sk = S.sanns_keygen(ctx, key_seed)
    db = S.sanns_encode_db(ctx, cu(coords), cu(perm))
    qids = cu(np.array([qid], dtype=np.uint64))
    ct_in = S.sanns_encrypt_query(ctx, sk, cu(q), enc_seed, qids)
    out_buf = torch.empty((1, K, 2, L, N), dtype=torch.uint64, device="cuda")
    tuned, _ = S.sanns_autotune_mac(ctx, db, ct_in, out_buf, reps=2)
    order = [tuned] + [v for v in range(len(S.sanns_mac_variants())) if v != tuned]
    runs = []
    for v in order:
        S.sanns_set_mac_variant(ctx, v)
        out, srv = S.sanns_distances(ctx, db, ct_in, mask_seed, qids)
        runs.append((v, out.cpu().numpy(), srv.cpu().numpy()))
    cli = S.sanns_decrypt_shares(ctx, sk, out, n, cu(q))
    # brute-force squared distances of every position, on the device
    pts = cu(coords).index_select(0, cu(perm.astype(np.int64)))
    brute = ((pts.int() - cu(q)[0].int()) ** 2).sum(1).long()
    t = ctx.query()["t"]
    rec_ok = bool(torch.equal((cli[0].long() + srv[0].long()) % t, brute))
    return ct_in.cpu().numpy(), runs, cli.cpu().numpy(), rec_ok


def _check_against_oracle(cfg, coords, perm, q, qid, key_seed, enc_seed, mask_seed, ct_in, runs, cli):
    N = cfg[0]
    n = len(perm)
    K = -(-n // N)
    O = Oracle(*cfg)
    s, s_hat = O.keygen(key_seed)
    assert np.array_equal(ct_in[0], O.encrypt(s_hat, q[0], enc_seed, qid))
    for k in sorted({0, K // 2, K - 1}):
        want_out, want_srv = O.distances(ct_in[0], coords, perm, mask_seed, qid, k0=k, k1=k + 1)
        cnt = len(want_srv)
        for v, out, srv in runs:
            assert np.array_equal(out[0, k], want_out[0]), (v, k)
            assert np.array_equal(srv[0, k * N:k * N + cnt], want_srv), (v, k)
        want_cli = O.decrypt_shares(want_out, s, q[0], cnt)
        assert np.array_equal(cli[0, k * N:k * N + cnt], want_cli), k


def test_full_size_linear_scan_matches_oracle_on_sampled_blocks():
    d = CFG[4]
    coords, perm, q = _inputs(N_POINTS, d)
    ct_in, runs, cli, rec_ok = _gpu_run(CFG, coords, perm, q, 7, 5, 6, 8)
    assert rec_ok   # every position: shares reconstruct the brute-force distance
    _check_against_oracle(CFG, coords, perm, q, 7, 5, 6, 8, ct_in, runs, cli)


C3 = (8192, 3, 60, 0, 96)
N_C3, B_C3 = 10_000_000, 64


def test_full_size_batched_matches_oracle_on_sampled_blocks():
    N, L, _, _, d = C3
    ctx = S.sanns_ctx_create(*C3)
    coords_d = inputs.mixture_coords_device(N_C3, d, 256, 12.0, 7)
    perm_d = inputs.permutation_device(N_C3, 8)
    db = S.sanns_encode_db(ctx, coords_d, perm_d)
    S.sanns_db_prepare_batched(ctx, db)
    q_d = inputs.mixture_coords_device(B_C3, d, 256, 12.0, 9, means_seed=7)
    qids = (torch.arange(B_C3, dtype=torch.int64) * 3 + 100).to(torch.uint64).cuda()
    sk = S.sanns_keygen(ctx, 10)
    ct = S.sanns_encrypt_query(ctx, sk, q_d, 11, qids)
    K = db.K
    out = torch.empty((B_C3, K, 2, L, N), dtype=torch.uint64, device="cuda")
    S.sanns_autotune_batched(ctx, db, ct, out, reps=1)
    out, srv = S.sanns_distances_batched(ctx, db, ct, 12, qids, out)
    S.sanns_device_status(ctx)
    # every query, whole, against the per-query path
    out_p = torch.empty((1, K, 2, L, N), dtype=torch.uint64, device="cuda")
    srv_p = torch.empty((1, N_C3), dtype=torch.uint32, device="cuda")
    for b in range(B_C3):
        S.sanns_distances(ctx, db, ct[b:b + 1], 12, qids[b:b + 1], out_p, srv_p)
        assert torch.equal(out_p[0], out[b]) and torch.equal(srv_p[0], srv[b]), b
    del out_p, srv_p
    # every position of every query: the shares reconstruct brute force
    cli = S.sanns_decrypt_shares(ctx, sk, out, N_C3, q_d)
    t = ctx.query()["t"]
    pts = coords_d.index_select(0, perm_d.view(torch.int32).long()).int()
    for b in range(B_C3):
        brute = ((pts - q_d[b].int()) ** 2).sum(1).long()
        assert torch.equal((cli[b].long() + srv[b].long()) % t, brute), b
    del pts
    # sampled queries and blocks against the oracle
    coords, perm = coords_d.cpu().numpy(), perm_d.cpu().numpy()
    q, qid_np = q_d.cpu().numpy(), qids.cpu().numpy()
    O = Oracle(*C3)
    s_, s_hat = O.keygen(10)
    for b in (0, 37, B_C3 - 1):
        ct_b = ct[b].cpu().numpy()
        assert np.array_equal(ct_b, O.encrypt(s_hat, q[b], 11, int(qid_np[b]))), b
        for k in (0, K // 2, K - 1):
            want_out, want_srv = O.distances(ct_b, coords, perm, 12, int(qid_np[b]), k0=k, k1=k + 1)
            cnt = len(want_srv)
            assert np.array_equal(out[b, k].cpu().numpy(), want_out[0]), (b, k)
            assert np.array_equal(srv[b, k * N:k * N + cnt].cpu().numpy(), want_srv), (b, k)
            want_cli = O.decrypt_shares(want_out, s_, q[b], cnt)
            assert np.array_equal(cli[b, k * N:k * N + cnt].cpu().numpy(), want_cli), (b, k)
