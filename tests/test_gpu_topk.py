"""GPU selection (plaintext meaning of Algorithms 1 and 2) against the oracle's
selection code, and the first configuration end to end: encrypted distances,
decryption, exact top-10, compared with a brute-force top-10."""
import numpy as np
import pytest
import torch

from oracle import select
from oracle.bfv import Oracle
from paper_1904_02033_b300 import inputs
from paper_1904_02033_b300 import sanns as S

pytestmark = pytest.mark.gpu


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def ctx():
    return S.sanns_ctx_create(256, 2, 40, 0, 4)


@pytest.mark.parametrize("n,spread", [(100_003, 50), (70_000, 1 << 24), (33, 5)])
@pytest.mark.parametrize("k", [1, 10, 32, 33, 88, 1024])   # > 32: the shared-memory sort path
def test_topk_matches_oracle(ctx, n, spread, k):
    t = ctx.query()["t"]
    rnd = np.random.default_rng(n + k)
    B = 3
    dist = rnd.integers(0, spread, size=(B, n)).astype(np.int64) % t   # many ties for small spread
    srv = rnd.integers(0, t, size=(B, n)).astype(np.int64)
    cli = (dist - srv) % t
    cli_d, srv_d = cu(cli.astype(np.uint32)), cu(srv.astype(np.uint32))
    if k > n:   # fewer elements than winners: rejected on the host, nothing launched
        for bins in (0, n):
            with pytest.raises(S.SannsError) as e:
                S.sanns_topk(ctx, cli_d, srv_d, k, bins)
            assert e.value.code == -1
        return
    pos = np.arange(n)
    for bins in sorted({0, max(k, n // 128), max(k, n // 7), n}):
        for shift in (0, 3):
            gd, gp = S.sanns_topk(ctx, cli_d, srv_d, k, bins, shift)
            gd, gp = gd.cpu().numpy(), gp.cpu().numpy()
            for b in range(B):
                ds = dist[b] >> shift
                if bins:
                    ov, oi = select.approx_topk_by_position(ds, pos, k, bins)
                    if bins * k <= 4_000_000:   # Algorithm 2 written out is O(l k)
                        assert ov == select.approx_topk(ds, pos, k, bins)[0]
                else:
                    ov, oi = select.exact_topk(ds, pos, k)
                assert gd[b].tolist() == ov and gp[b].tolist() == oi, (bins, shift, b)


def test_topk_rejects_bad_arguments(ctx):
    z = torch.zeros((1, 100), dtype=torch.uint32, device="cuda")
    for k, bins, shift in [(0, 0, 0), (1025, 0, 0), (10, 5, 0), (10, 101, 0), (101, 0, 0), (10, 0, 32)]:
        with pytest.raises(S.SannsError):
            S.sanns_topk(ctx, z, z, k, bins, shift)


def test_first_configuration_end_to_end_top10():
    # n = 4096, d = 32 uniform coordinates, N = 4096, two 54-bit primes
    cfg = (4096, 2, 54, 0, 32)
    n, d, k = 4096, 32, 10
    ctx = S.sanns_ctx_create(*cfg)
    coords = inputs.uniform_coords(n, d, 0)
    perm = inputs.permutation(n, 1)
    q = inputs.uniform_coords(1, d, 2)
    qids = cu(np.array([0], dtype=np.uint64))
    sk = S.sanns_keygen(ctx, 0)
    db = S.sanns_encode_db(ctx, cu(coords), cu(perm))
    ct = S.sanns_encrypt_query(ctx, sk, cu(q), 0, qids)
    out, srv = S.sanns_distances(ctx, db, ct, 0, qids)
    cli = S.sanns_decrypt_shares(ctx, sk, out, n, cu(q))
    gd, gp = S.sanns_topk(ctx, cli, srv, k)
    brute = np.sum((coords[perm].astype(np.int64) - q[0].astype(np.int64)) ** 2, axis=1)
    ev, ep = select.exact_topk(brute, np.arange(n), k)
    assert gd.cpu().numpy()[0].tolist() == ev and gp.cpu().numpy()[0].tolist() == ep
    # positions name points of the server's permuted order
    ids = perm[gp.cpu().numpy()[0]]
    assert np.array_equal(np.sort(np.sum((coords[ids].astype(np.int64) - q[0]) ** 2, axis=1)),
                          np.array(ev))


@pytest.mark.parametrize("k,bins", [(10, 0), (10, 40), (40, 0), (40, 64)])
def test_topk_segments_matches_oracle(ctx, k, bins):
    # ragged lists: empty, shorter than k, shorter than the bins, long ones;
    # increasing offsets with gaps in the client shares, a shuffled order in
    # the server shares
    t = ctx.query()["t"]
    rnd = np.random.default_rng(k * 7 + bins)
    lens = np.array([0, 3, k - 1, k, bins + 5, 999, 70_001, 5, 20_000], dtype=np.int64)
    B = len(lens)
    gaps = rnd.integers(0, 50, size=B)
    co = np.concatenate([[0], np.cumsum(lens + gaps)[:-1]]) + gaps
    order = rnd.permutation(B)
    so = np.zeros(B, dtype=np.int64)
    so[order] = np.concatenate([[0], np.cumsum(lens[order] + 3)[:-1]])
    srv = rnd.integers(0, t, size=int(so.max() + lens.max() + 10)).astype(np.int64)
    cli = rnd.integers(0, t, size=int(co[-1] + lens[-1] + 10)).astype(np.int64)
    want = []
    for b in range(B):
        v = rnd.integers(0, 300, size=lens[b]).astype(np.int64)       # many ties
        cli[co[b]:co[b] + lens[b]] = (v - srv[so[b]:so[b] + lens[b]]) % t
        want.append(v)
    for shift in (0, 2):
        gd, gp = S.sanns_topk_segments(ctx, cu(cli.astype(np.uint32)), cu(srv.astype(np.uint32)),
                                       co, so, lens, k, bins, shift)
        gd, gp = gd.cpu().numpy(), gp.cpu().numpy()
        for b in range(B):
            ds = want[b] >> shift
            n = int(lens[b])
            pos = np.arange(n)
            lb = min(bins, n)
            if bins and lb >= 1:
                ov, oi = select.approx_topk_by_position(ds, pos, min(k, lb), lb)
            else:
                ov, oi = select.exact_topk(ds, pos, min(k, n))
            fill = k - len(ov)
            assert gd[b].tolist() == ov + [2 ** 32 - 1] * fill, (b, shift)
            assert gp[b].tolist() == oi + [-1] * fill, (b, shift)


def test_topk_segments_rejects_bad_arguments(ctx):
    z = torch.zeros(100, dtype=torch.uint32, device="cuda")
    one = np.array([0])
    for k, bins, shift, ln in [(0, 0, 0, 10), (1025, 0, 0, 10), (10, 5, 0, 10), (10, 0, 32, 10),
                               (10, 0, 0, 2 ** 32)]:
        with pytest.raises((S.SannsError, AssertionError)):
            S.sanns_topk_segments(ctx, z, z, one, one, np.array([ln]), k, bins, shift)


def test_topk_segments_per_list_k_and_bins(ctx):
    # every list its own winners and bins (the centre groups of Algorithm 4)
    t = ctx.query()["t"]
    rnd = np.random.default_rng(5)
    lens = np.array([500, 37, 9000, 3, 0, 64], dtype=np.int64)
    ks = np.array([7, 33, 50, 2, 4, 1])
    for approx in (False, True):
        ls = np.array([40, 33, 300, 2, 8, 64]) if approx else None
        co = np.concatenate([[0], np.cumsum(lens)[:-1]])
        v = rnd.integers(0, 100, size=int(lens.sum())).astype(np.int64)
        srv = rnd.integers(0, t, size=len(v)).astype(np.int64)
        cli = (v - srv) % t
        kmax = int(ks.max())
        gd, gp = S.sanns_topk_segments(ctx, cu(cli.astype(np.uint32)), cu(srv.astype(np.uint32)), co, co,
                                       lens, kmax, int(ls.max()) if approx else 0, 1, k_seg=ks,
                                       bins_seg=ls)
        gd, gp = gd.cpu().numpy(), gp.cpu().numpy()
        for b in range(len(lens)):
            ds = v[co[b]:co[b] + lens[b]] >> 1
            n = int(lens[b])
            kb = min(int(ks[b]), n)
            if approx and n:
                lb = min(int(ls[b]), n)
                ov, oi = select.approx_topk_by_position(ds, np.arange(n), min(int(ks[b]), lb), lb)
            else:
                ov, oi = select.exact_topk(ds, np.arange(n), kb)
            fill = kmax - len(ov)
            assert gd[b].tolist() == ov + [2 ** 32 - 1] * fill, (approx, b)
            assert gp[b].tolist() == oi + [-1] * fill, (approx, b)
    with pytest.raises(S.SannsError):   # a list's k above the call's k
        S.sanns_topk_segments(ctx, cu(cli.astype(np.uint32)), cu(srv.astype(np.uint32)), co, co, lens, 10,
                              0, 0, k_seg=ks)
