"""GPU parity: every output of the CUDA path, called through the C ABI, is
compared element by element with the CPU oracle on the same seeded inputs.
All comparisons are bit-exact (integer arithmetic throughout)."""
import numpy as np
import pytest
import torch

from oracle.bfv import Oracle
from paper_1904_02033_b300 import inputs
from paper_1904_02033_b300 import sanns as S

pytestmark = pytest.mark.gpu

_ORACLES = {}


def oracle(N, L, bits, rule, d, b_c=8):
    key = (N, L, bits, rule, d)
    if key not in _ORACLES:
        _ORACLES[key] = Oracle(N, L, bits, rule, d)
    return _ORACLES[key]


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def np_(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


CONFIGS = [
    # N, L, bits, t_rule, d
    (64, 1, 30, 0, 3),
    (256, 2, 40, 0, 5),
    (256, 3, 60, 1, 17),
    (4096, 2, 54, 0, 32),
    (8192, 3, 60, 0, 7),
    (16384, 4, 60, 0, 5),   # the largest ring and prime count the API accepts
]


@pytest.mark.parametrize("cfg", CONFIGS)
def test_context_constants_match_oracle(cfg):
    ctx = S.sanns_ctx_create(*cfg)
    O = oracle(*cfg)
    info = ctx.query()
    assert info["q"] == O.P.q
    assert info["psi"] == O.P.psi
    assert info["t"] == O.P.t
    assert info["delta"] == O.P.delta_mod_q


@pytest.mark.parametrize("cfg", CONFIGS)
def test_ntt_forward_inverse_match_oracle(cfg):
    N, L = cfg[0], cfg[1]
    ctx = S.sanns_ctx_create(*cfg)
    O = oracle(*cfg)
    rnd = np.random.default_rng(N + L)
    cnt = 3
    a = np.zeros((cnt, L, N), dtype=np.uint64)
    for j in range(L):
        a[:, j] = rnd.integers(0, int(O.q[j]), size=(cnt, N), dtype=np.uint64)
    a[1, 0] = O.q[0] - 1   # all q - 1
    a[2, 0] = 0
    a[2, 0, N // 3] = 1
    t = cu(a)
    S.sanns_ntt(ctx, t)
    f = np_(t)
    for g in range(cnt):
        for j in range(L):
            assert np.array_equal(f[g, j], O.ntt(a[g, j], j))
    S.sanns_ntt(ctx, t, inverse=True)
    assert np.array_equal(np_(t), a)


@pytest.mark.parametrize("cfg", CONFIGS)
def test_keygen_matches_oracle(cfg):
    ctx = S.sanns_ctx_create(*cfg)
    O = oracle(*cfg)
    sk = S.sanns_keygen(ctx, seed=5)
    s, s_hat = S.sanns_sk_export(sk)
    os_, os_hat = O.keygen(5)
    assert np.array_equal(np_(s), os_)
    assert np.array_equal(np_(s_hat), os_hat)


@pytest.mark.parametrize("cfg", CONFIGS)
def test_encrypt_matches_oracle(cfg):
    ctx = S.sanns_ctx_create(*cfg)
    O = oracle(*cfg)
    d = cfg[4]
    sk = S.sanns_keygen(ctx, seed=1)
    _, os_hat = O.keygen(1)
    B = 2
    q = inputs.uniform_coords(B, d, 3)
    q[0, 0] = 0
    q[1, -1] = 255
    qids = np.array([7, 2 ** 40 + 3], dtype=np.uint64)
    ct = S.sanns_encrypt_query(ctx, sk, cu(q), seed=9, qids=cu(qids))
    got = np_(ct)
    for b in range(B):
        want = O.encrypt(os_hat, q[b], seed=9, qid=int(qids[b]))
        assert np.array_equal(got[b], want)


@pytest.mark.parametrize("cfg,n", [(CONFIGS[1], 600), (CONFIGS[2], 256), (CONFIGS[3], 4096),
                                   (CONFIGS[4], 8192 * 2 + 77), (CONFIGS[0], 1)])
def test_encode_db_matches_oracle(cfg, n):
    ctx = S.sanns_ctx_create(*cfg)
    O = oracle(*cfg)
    d = cfg[4]
    coords = inputs.uniform_coords(n + 5, d, 11)
    perm = inputs.permutation(n + 5, 12)[:n]
    db = S.sanns_encode_db(ctx, cu(coords), cu(perm))
    pt, norms = S.sanns_db_export(db)
    opt, onorms = O.encode_db(coords, perm)
    assert np.array_equal(np_(pt), opt)
    assert np.array_equal(np_(norms), onorms)


def _pipeline(cfg, n, B, seed, perm=True):
    N, L, bits, rule, d = cfg
    ctx = S.sanns_ctx_create(*cfg)
    coords = inputs.uniform_coords(n, d, seed)
    pm = inputs.permutation(n, seed + 1) if perm else None
    q = inputs.uniform_coords(B, d, seed + 2)
    qids = np.arange(100, 100 + B, dtype=np.uint64)
    sk = S.sanns_keygen(ctx, seed + 3)
    db = S.sanns_encode_db(ctx, cu(coords), cu(pm) if perm else None)
    ct_in = S.sanns_encrypt_query(ctx, sk, cu(q), seed + 4, cu(qids))
    ct_out, srv = S.sanns_distances(ctx, db, ct_in, seed + 5, cu(qids))
    cli = S.sanns_decrypt_shares(ctx, sk, ct_out, n, cu(q))
    return dict(ctx=ctx, coords=coords, pm=pm, q=q, qids=qids, ct_in=np_(ct_in),
                ct_out=np_(ct_out), srv=np_(srv), cli=np_(cli), seed=seed)


@pytest.mark.parametrize("cfg,n,B", [
    # a single 60-bit prime: Delta = floor(q / t) ~ 2^36 exceeds twice the
    # noise, whose largest term is (Q mod t) floor(M / t) <= t d 255 ~ 2^33.6
    # for the plaintext product M = sum_i m_i g_i (smaller primes are not
    # decryptable at t ~ 2^24)
    ((64, 1, 60, 0, 3), 1, 1),
    (CONFIGS[1], 600, 2),         # three blocks, ragged tail, two queries
    (CONFIGS[2], 700, 1),         # d = 17 (not a multiple of the 16-dim fold), t = 2^b_d
    (CONFIGS[3], 4096, 1),        # the one-block N = 4096 configuration
    (CONFIGS[4], 8192 * 3 - 5, 1),  # N = 8192, three 60-bit primes, ragged
    # more than two waves of epilogue blocks (B K 2 L > 2 x 3 x SMs): the fused
    # INTT + mask kernel, with the padding positions of the last block
    (CONFIGS[1], 256 * 60 - 17, 8),
    (CONFIGS[4], 8192 * 38 - 1000, 4),
    (CONFIGS[5], 16384 + 77, 2),    # N = 16384, four 60-bit primes, ragged, a query pair
])
def test_distances_match_oracle_bit_exact(cfg, n, B):
    r = _pipeline(cfg, n, B, seed=n % 97)
    O = oracle(*cfg)
    _, os_hat = O.keygen(r["seed"] + 3)
    os_, _ = O.keygen(r["seed"] + 3)
    for b in range(B):
        assert np.array_equal(r["ct_in"][b], O.encrypt(os_hat, r["q"][b], r["seed"] + 4,
                                                       int(r["qids"][b])))
        out, srv = O.distances(r["ct_in"][b], r["coords"], r["pm"], r["seed"] + 5,
                               int(r["qids"][b]))
        assert np.array_equal(r["ct_out"][b], out)
        assert np.array_equal(r["srv"][b], srv)
        cli = O.decrypt_shares(out, os_, r["q"][b], n)
        assert np.array_equal(r["cli"][b], cli)
        order = r["pm"] if r["pm"] is not None else np.arange(n)
        brute = np.sum((r["coords"][order].astype(np.int64) - r["q"][b].astype(np.int64)) ** 2,
                       axis=1)
        assert np.array_equal((r["cli"][b].astype(np.int64) + r["srv"][b]) % O.t, brute)


@pytest.mark.parametrize("cfg,n,B", [
    ((1024, 2, 40, 0, 9), 1024 * 3 - 7, 2),    # quarters of 256: radix-4 passes only
    ((2048, 3, 60, 1, 6), 2048 * 2 + 1, 1),    # quarters of 512: a radix-2 stage too; t = 2^b_d
])
def test_few_polynomials_on_clusters_match_oracle(cfg, n, B):
    """At most 37 response polynomials (B K 2 L): the epilogue runs each
    polynomial on a cluster of four CTAs and draws the mask itself; the N =
    4096, 8192 and 16384 cases above take the same path."""
    K = -(-n // cfg[0])
    assert B * K * 2 * cfg[1] * 4 <= S.sanns_device_sms()
    test_distances_match_oracle_bit_exact(cfg, n, B)


def test_max_dimension_and_identity_perm():
    cfg = (64, 2, 40, 0, 224)
    r = _pipeline(cfg, 130, 1, seed=3, perm=False)
    O = oracle(*cfg)
    os_, _ = O.keygen(6)
    out, srv = O.distances(r["ct_in"][0], r["coords"], None, 8, int(r["qids"][0]))
    assert np.array_equal(r["ct_out"][0], out)
    assert np.array_equal(r["srv"][0], srv)


def test_bad_permutation_rejected():
    ctx = S.sanns_ctx_create(256, 2, 40, 0, 5)
    coords = cu(inputs.uniform_coords(10, 5, 1))
    perm = cu(np.array([0, 3, 10], dtype=np.uint32))
    with pytest.raises(S.SannsError) as e:
        S.sanns_encode_db(ctx, coords, perm)
    assert e.value.code == -1


@pytest.mark.parametrize("cfg,n", [((8192, 3, 60, 0, 7), 8192 * 4 + 3), ((4096, 2, 54, 0, 128), 4096 * 5),
                                   ((256, 2, 40, 0, 200), 1000)])
def test_every_mac_variant_matches_oracle(cfg, n):
    ctx = S.sanns_ctx_create(*cfg)
    O = oracle(*cfg)
    d = cfg[4]
    coords = inputs.uniform_coords(n, d, 5)
    sk = S.sanns_keygen(ctx, 1)
    q = inputs.uniform_coords(1, d, 6)
    qids = cu(np.array([3], dtype=np.uint64))
    db = S.sanns_encode_db(ctx, cu(coords))
    ct_in = S.sanns_encrypt_query(ctx, sk, cu(q), 2, qids)
    pt, _ = O.encode_db(coords, None)
    want = O.mac(np_(ct_in)[0], pt)
    names = S.sanns_mac_variants()
    assert len(names) >= 2
    for v in range(len(names)):
        S.sanns_set_mac_variant(ctx, v)
        acc = S.sanns_distances_mac(ctx, db, ct_in)
        assert np.array_equal(np_(acc)[0], want), names[v]
    best, ms = S.sanns_autotune_mac(ctx, db, ct_in, acc, reps=1)
    assert 0 <= best < len(names) and all(m > 0 for m in ms)


@pytest.mark.parametrize("cfg,n,B", [((8192, 3, 60, 0, 7), 8192 * 2 + 5, 3), ((256, 2, 40, 0, 200), 700, 4),
                                     ((256, 2, 40, 0, 224), 300, 5)])
def test_multi_query_mac_matches_oracle(cfg, n, B):
    # calls with B >= 2 run the pair variants (two queries per pass over the
    # database, a lone last query for odd B), also at the largest d
    ctx = S.sanns_ctx_create(*cfg)
    O = oracle(*cfg)
    d = cfg[4]
    coords = inputs.uniform_coords(n, d, 8)
    sk = S.sanns_keygen(ctx, 2)
    q = inputs.uniform_coords(B, d, 9)
    qids = cu(np.arange(B, dtype=np.uint64) + 11)
    db = S.sanns_encode_db(ctx, cu(coords))
    ct_in = S.sanns_encrypt_query(ctx, sk, cu(q), 3, qids)
    pt, _ = O.encode_db(coords, None)
    ct_np = np_(ct_in)
    want = [O.mac(ct_np[b], pt) for b in range(B)]
    for v in range(len(S.sanns_mac_variants())):
        S.sanns_set_mac_variant(ctx, v)
        acc = np_(S.sanns_distances_mac(ctx, db, ct_in))
        for b in range(B):
            assert np.array_equal(acc[b], want[b]), (S.sanns_mac_variants()[v], b)


def test_db_import_of_the_oracle_encoding_equals_encode_db():
    """A database imported from the oracle's plaintexts and norms computes
    the same responses as the one the library encodes itself; a residue not
    below its prime is rejected and nothing is created."""
    cfg = (256, 2, 40, 0, 5)
    N, L, bits, rule, d = cfg
    n = 3 * N - 11
    ctx = S.sanns_ctx_create(*cfg)
    O = oracle(*cfg)
    coords = inputs.uniform_coords(n, d, 71)
    perm = inputs.permutation(n, 72)
    pt, norms = O.encode_db(coords, perm)
    db_imp = S.sanns_db_import(ctx, n, cu(pt), cu(norms))
    db_enc = S.sanns_encode_db(ctx, cu(coords), cu(perm))
    sk = S.sanns_keygen(ctx, 73)
    qids = cu(np.array([5], dtype=np.uint64))
    ct = S.sanns_encrypt_query(ctx, sk, cu(inputs.uniform_coords(1, d, 74)), 75, qids)
    a_out, a_srv = S.sanns_distances(ctx, db_imp, ct, 76, qids)
    b_out, b_srv = S.sanns_distances(ctx, db_enc, ct, 76, qids)
    assert torch.equal(a_out, b_out) and torch.equal(a_srv, b_srv)
    ept, enorms = S.sanns_db_export(db_imp)
    assert np.array_equal(np_(ept), pt) and np.array_equal(np_(enorms), norms)
    # norms are only ever used mod t: imported ones at or above t are stored
    # reduced and give the same responses
    db_big = S.sanns_db_import(ctx, n, cu(pt), cu(norms + np.uint32(O.t)))
    c_out, c_srv = S.sanns_distances(ctx, db_big, ct, 76, qids)
    assert torch.equal(c_out, b_out) and torch.equal(c_srv, b_srv)
    assert np.array_equal(np_(S.sanns_db_export(db_big)[1]), norms)
    bad = pt.copy()
    bad[1, 1, 2, 7] = O.q[1]
    with pytest.raises(S.SannsError) as e:
        S.sanns_db_import(ctx, n, cu(bad), cu(norms))
    assert e.value.code == -1


def test_mac_sm_cap_and_two_stream_pipeline_keep_results():
    """The MAC's grid capped to fewer SMs, and consecutive queries pipelined
    over two streams (MAC of one query beside the INTT + mask of the
    previous, responses double-buffered), give the single-stream results."""
    cfg = (4096, 2, 54, 0, 16)
    N, L, bits, rule, d = cfg
    n = 4096 * 7 - 5
    ctx = S.sanns_ctx_create(*cfg)
    db = S.sanns_encode_db(ctx, cu(inputs.uniform_coords(n, d, 81)), cu(inputs.permutation(n, 82)))
    sk = S.sanns_keygen(ctx, 83)
    B = 6
    qids = cu(np.arange(B, dtype=np.uint64))
    ct = S.sanns_encrypt_query(ctx, sk, cu(inputs.uniform_coords(B, d, 84)), 85, qids)
    want = [S.sanns_distances(ctx, db, ct[b:b + 1], 86, qids[b:b + 1]) for b in range(B)]
    with pytest.raises(S.SannsError):
        S.sanns_set_mac_sms(ctx, -1)
    for cap in (7, 100):
        S.sanns_set_mac_sms(ctx, cap)
        s_mac, s_fin = torch.cuda.Stream(), torch.cuda.Stream()
        outs = [torch.empty_like(want[0][0]) for _ in range(2)]
        srvs = [torch.empty_like(want[0][1]) for _ in range(2)]
        got = []
        fin = [None] * B
        for b in range(B):
            if b >= 2:
                s_mac.wait_event(fin[b - 2])
                torch.cuda.current_stream().wait_event(fin[b - 2])
            S.sanns_distances_mac(ctx, db, ct[b:b + 1], outs[b % 2], stream=s_mac)
            ev = torch.cuda.Event()
            ev.record(s_mac)
            s_fin.wait_event(ev)
            S.sanns_distances_finish(ctx, db, outs[b % 2], 86, qids[b:b + 1], srvs[b % 2], stream=s_fin)
            fin[b] = torch.cuda.Event()
            fin[b].record(s_fin)
            s_fin.synchronize()
            got.append((outs[b % 2].clone(), srvs[b % 2].clone()))
        torch.cuda.synchronize()
        for b in range(B):
            assert torch.equal(got[b][0], want[b][0]) and torch.equal(got[b][1], want[b][1]), (cap, b)
    S.sanns_set_mac_sms(ctx, 0)


@pytest.mark.parametrize("batched", [False, True])
def test_norms_above_t_with_few_bits_per_coordinate(batched):
    """The paper's t = 2^(2 b_c + ceil(log2 d)) with b_c = 6 bits per
    coordinate is below the norms of 8-bit coordinates, so ||p||^2 + r is
    reduced mod t the general way: responses and shares still equal the
    oracle's (same b_c), and the shares reconstruct the distances mod t."""
    cfg = (256, 2, 40, 1, 5)
    n, B = 700, 2
    ctx = S.sanns_ctx_create(*cfg, b_c=6)
    O = Oracle(*cfg, b_c=6)
    assert O.t == 2 ** 15 < 5 * 255 ** 2
    coords = inputs.uniform_coords(n, cfg[4], 81)
    coords[:9] = 255
    perm = inputs.permutation(n, 82)
    q = inputs.uniform_coords(B, cfg[4], 83)
    qids = np.array([7, 8], dtype=np.uint64)
    sk = S.sanns_keygen(ctx, 84)
    db = S.sanns_encode_db(ctx, cu(coords), cu(perm))
    ct = S.sanns_encrypt_query(ctx, sk, cu(q), 85, cu(qids))
    if batched:
        S.sanns_db_prepare_batched(ctx, db)
        out, srv = S.sanns_distances_batched(ctx, db, ct, 86, cu(qids))
    else:
        out, srv = S.sanns_distances(ctx, db, ct, 86, cu(qids))
    cli = S.sanns_decrypt_shares(ctx, sk, out, n, cu(q))
    s_, _ = O.keygen(84)
    for b in range(B):
        want_out, want_srv = O.distances(np_(ct)[b], coords, perm, 86, int(qids[b]))
        assert np.array_equal(np_(out)[b], want_out)
        assert np.array_equal(np_(srv)[b], want_srv)
        assert np.array_equal(np_(cli)[b], O.decrypt_shares(want_out, s_, q[b], n))
        brute = np.sum((coords[perm].astype(np.int64) - q[b].astype(np.int64)) ** 2, axis=1)
        assert np.array_equal((np_(cli)[b].astype(np.int64) + np_(srv)[b]) % O.t, brute % O.t)
