"""GPU parity of the batched tensor-core MAC: its ciphertexts must be
bit-identical to the plain per-query path and to the oracle."""
import numpy as np
import pytest
import torch

from oracle.bfv import Oracle
from paper_1904_02033_b300 import inputs
from paper_1904_02033_b300 import sanns as S

pytestmark = pytest.mark.gpu


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


TILES = [0, 1, 2, 3, 4, 5, 6, 7, 8]
TILE_IDS = ["tile128", "tile256pair", "tile128tma", "tile256pairtma", "tile128tma_cl2",
            "tile128tma_cl4", "tile128quad", "tile128quad_cl2", "tile256pairquad"]


@pytest.mark.parametrize("tile", TILES, ids=TILE_IDS)
@pytest.mark.parametrize("cfg,n,B", [
    ((256, 2, 40, 0, 16), 700, 3),          # one ragged N tile, partial M tile
    ((256, 3, 60, 0, 96), 256 * 300, 9),    # two N tiles (K = 300), three M tiles
    ((64, 2, 50, 0, 13), 64 * 5 - 1, 1),    # d not a multiple of 8, B = 1
    ((8192, 3, 60, 0, 128), 8192 * 2 + 5, 2),  # d = 128: partial sums up to 2^24
    ((256, 2, 60, 0, 24), 256 * 600 - 3, 20),  # 40 query rows: two query tiles, K = 600
    ((256, 2, 40, 0, 16), 256 * 200 - 5, 6),   # two 128-block tiles: one cluster of 2
    ((256, 2, 60, 0, 24), 256 * 500 - 7, 20),  # four tiles, two query tiles: clusters of 2 and 4
])
def test_batched_equals_plain_and_oracle(cfg, n, B, tile):
    N, L, bits, rule, d = cfg
    ctx = S.sanns_ctx_create(*cfg)
    S.sanns_batched_tune(ctx, tile=tile)
    rnd = np.random.default_rng(n + B)
    coords = rnd.integers(0, 256, size=(n, d), dtype=np.uint8)
    coords[: min(n, 50)] = 255      # extreme digits on the database side
    perm = inputs.permutation(n, 3)
    q = rnd.integers(0, 256, size=(B, d), dtype=np.uint8)
    qids = cu(np.arange(10, 10 + B, dtype=np.uint64))
    sk = S.sanns_keygen(ctx, 4)
    db = S.sanns_encode_db(ctx, cu(coords), cu(perm))
    S.sanns_db_prepare_batched(ctx, db)
    ct_in = S.sanns_encrypt_query(ctx, sk, cu(q), 5, qids)
    plain_out, plain_srv = S.sanns_distances(ctx, db, ct_in, 6, qids)
    acc_plain = S.sanns_distances_mac(ctx, db, ct_in)
    acc_batch = S.sanns_distances_batched_mac(ctx, db, ct_in)
    S.sanns_device_status(ctx)
    assert torch.equal(acc_batch.cpu(), acc_plain.cpu())
    bout, bsrv = S.sanns_distances_batched(ctx, db, ct_in, 6, qids)
    S.sanns_device_status(ctx)
    assert torch.equal(bout.cpu(), plain_out.cpu())
    assert torch.equal(bsrv.cpu(), plain_srv.cpu())
    if N <= 256:
        O = Oracle(*cfg)
        out0, srv0 = O.distances(ct_in.cpu().numpy()[0], coords, perm, 6, 10)
        assert np.array_equal(bout.cpu().numpy()[0], out0)
        s, _ = O.keygen(4)
        cli = O.decrypt_shares(out0, s, q[0], n)
        brute = np.sum((coords[perm].astype(np.int64) - q[0].astype(np.int64)) ** 2, axis=1)
        assert np.array_equal((cli.astype(np.int64) + srv0) % O.t, brute)


@pytest.mark.parametrize("tile", [2, 6, 7, 8])
def test_many_slot_ranges_equal_one(tile):
    """A 3 MiB scratch cap splits N = 256 slots into 22 ranges of 12 (the
    last of 4), each with its own query expansion and MAC launch; the
    responses equal the per-query path's, as with one range, and the scratch
    the library reports is one range's."""
    cfg = (256, 2, 60, 0, 24)
    n, B = 256 * 512 - 7, 20          # four 128-block tiles: tile 7 runs in clusters of 2
    ctx = S.sanns_ctx_create(*cfg)
    rnd = np.random.default_rng(31)
    coords = rnd.integers(0, 256, size=(n, cfg[4]), dtype=np.uint8)
    q = rnd.integers(0, 256, size=(B, cfg[4]), dtype=np.uint8)
    qids = cu(np.arange(B, dtype=np.uint64))
    sk = S.sanns_keygen(ctx, 32)
    db = S.sanns_encode_db(ctx, cu(coords), cu(inputs.permutation(n, 33)))
    S.sanns_db_prepare_batched(ctx, db)
    ct_in = S.sanns_encrypt_query(ctx, sk, cu(q), 34, qids)
    acc_plain = S.sanns_distances_mac(ctx, db, ct_in)
    S.sanns_batched_tune(ctx, scratch_mib=3, tile=tile)
    per_slot = cfg[1] * 2 * B * 24 * 8 * 16     # fp16 digit rows of one slot, every prime
    assert S.sanns_distances_scratch_bytes(ctx, B, True) == 12 * per_slot
    acc_b = S.sanns_distances_batched_mac(ctx, db, ct_in)
    S.sanns_device_status(ctx)
    assert torch.equal(acc_b.cpu(), acc_plain.cpu())
    S.sanns_batched_tune(ctx, scratch_mib=4096, tile=tile)
    assert S.sanns_distances_scratch_bytes(ctx, B, True) == 256 * per_slot
    acc_1 = S.sanns_distances_batched_mac(ctx, db, ct_in)
    S.sanns_device_status(ctx)
    assert torch.equal(acc_1.cpu(), acc_plain.cpu())


@pytest.mark.parametrize("tile", TILES, ids=TILE_IDS)
def test_sm_cap_keeps_batched_results(tile):
    """The MAC SM cap bounds the tensor-core path's persistent grid too (one
    CTA, pair or cluster at the smallest caps, an odd cap for the clusters of
    2 and 4); the responses equal the per-query path's at every cap."""
    cfg = (256, 2, 60, 0, 24)
    n, B = 256 * 512 - 7, 12
    ctx = S.sanns_ctx_create(*cfg)
    rnd = np.random.default_rng(41)
    coords = rnd.integers(0, 256, size=(n, cfg[4]), dtype=np.uint8)
    q = rnd.integers(0, 256, size=(B, cfg[4]), dtype=np.uint8)
    sk = S.sanns_keygen(ctx, 42)
    db = S.sanns_encode_db(ctx, cu(coords), cu(inputs.permutation(n, 43)))
    S.sanns_db_prepare_batched(ctx, db)
    ct_in = S.sanns_encrypt_query(ctx, sk, cu(q), 44, cu(np.arange(B, dtype=np.uint64)))
    acc_plain = S.sanns_distances_mac(ctx, db, ct_in).cpu()
    S.sanns_batched_tune(ctx, tile=tile)
    for cap in (1, 2, 7, 100, 0):
        S.sanns_set_mac_sms(ctx, cap)
        acc_b = S.sanns_distances_batched_mac(ctx, db, ct_in)
        S.sanns_device_status(ctx)
        assert torch.equal(acc_b.cpu(), acc_plain), cap


def test_batched_needs_prepare_and_small_d():
    ctx = S.sanns_ctx_create(256, 2, 40, 0, 200)
    db = S.sanns_encode_db(ctx, cu(inputs.uniform_coords(300, 200, 1)))
    with pytest.raises(S.SannsError):
        S.sanns_db_prepare_batched(ctx, db)
    ct = torch.zeros((1, 200, 2, 2, 256), dtype=torch.uint64, device="cuda")
    with pytest.raises(S.SannsError):
        S.sanns_distances_batched_mac(ctx, db, ct)


def test_batched_autotune_keeps_results_identical():
    cfg = (256, 2, 40, 0, 16)
    n, B = 256 * 40 + 7, 5
    ctx = S.sanns_ctx_create(*cfg)
    coords = inputs.uniform_coords(n, cfg[4], 21)
    q = inputs.uniform_coords(B, cfg[4], 22)
    qids = cu(np.arange(B, dtype=np.uint64))
    sk = S.sanns_keygen(ctx, 23)
    db = S.sanns_encode_db(ctx, cu(coords), cu(inputs.permutation(n, 24)))
    S.sanns_db_prepare_batched(ctx, db)
    ct_in = S.sanns_encrypt_query(ctx, sk, cu(q), 25, qids)
    out = torch.empty((B, db.K, 2, 2, 256), dtype=torch.uint64, device="cuda")
    idx, ms = S.sanns_autotune_batched(ctx, db, ct_in, out, reps=1)
    assert 0 <= idx < len(S.BATCHED_CONFIGS) and len(ms) == len(S.BATCHED_CONFIGS)
    assert all(m > 0 for m in ms)
    acc_plain = S.sanns_distances_mac(ctx, db, ct_in)
    assert torch.equal(out.cpu(), acc_plain.cpu())
    acc_b = S.sanns_distances_batched_mac(ctx, db, ct_in)
    S.sanns_device_status(ctx)
    assert torch.equal(acc_b.cpu(), acc_plain.cpu())


def test_measured_tensor_rates_rank_the_instruction_families():
    """The library's rate probe: the tcgen05 fp16 MMA the batched kernel uses
    is faster than the legacy fp16 mma.sync, which is faster per operation
    than the legacy s8 mma.sync (the only INT8 tensor instruction on sm_103a)."""
    ctx = S.sanns_ctx_create(256, 2, 40, 0, 8)
    r = S.sanns_measure_mma_rates(ctx)
    assert r["tcgen05_f16_tflops"] > r["mma_sync_f16_tflops"] > r["mma_sync_s8_tops"] > 0
    # sanity bound: no more than the nominal dense fp16 peak plus margin
    assert r["tcgen05_f16_tflops"] < 3000


def _balanced_digits(v: int) -> list:
    """The eight balanced base-256 digits (each in [-128, 127]) of v < 2^62."""
    out = []
    for _ in range(8):
        t = v & 255
        v >>= 8
        if t >= 128:
            t -= 256
            v += 1
        out.append(t)
    assert v == 0
    return out


def _edge_query_value(q: int, V: int, d: int):
    """A residue A mod q whose multiples X_b = A 256^b mod q (b < 7) all have
    a digit near -128 at one position a, so that with the database residue V
    (seven digits -128) the digit sum S_a = d sum_b x_{b,a} v_b comes close to
    the 2^24 bound.  Starts from bytes 0x80 at the bit offsets where
    floor(A 2^(8b) / q) mod 256 is taken (q = 1 mod 256) and searches the free
    bits; returns (A, max_a |S_a|)."""
    v = _balanced_digits(V)
    base = sum(0x80 << off for off in (12, 20, 28, 36, 44, 52)) | 0x80
    best = (None, -1)
    for free in range(16):
        for tweak in range(-3, 4):
            A = (base | (free << 8)) + (tweak << 12)
            if not 0 <= A < q:
                continue
            xs = [_balanced_digits(A * pow(256, b, q) % q) for b in range(8)]
            mag = max(abs(d * sum(xs[b][a] * v[b] for b in range(8))) for a in range(8))
            if mag > best[1]:
                best = (A, mag)
    return best


@pytest.mark.parametrize("tile", TILES, ids=TILE_IDS)
def test_batched_exact_at_the_fp32_digit_sum_edge(tile):
    """Worst-case digits on both sides at d = 128: every database residue is
    V = 0x7F7F7F7F7F7F80 (digits -128 x 7, then 1) and every query residue
    a searched A_j whose multiples carry digits near -128, so the exact digit
    sums reach most of the 2^24 range fp32 holds exactly.  The MAC result is
    then sum_i A_j V = d A_j V mod q_j at every (query, block, component,
    slot), a closed form checked element by element."""
    N, L, bits, d = 256, 3, 60, 128
    ctx = S.sanns_ctx_create(N, L, bits, 0, d)
    S.sanns_batched_tune(ctx, tile=tile)
    qs = ctx.query()["q"]
    V = 0x7F7F7F7F7F7F80
    assert _balanced_digits(V) == [-128] * 7 + [1]
    A, mags = [], []
    for j in range(L):
        a, mag = _edge_query_value(int(qs[j]), V, d)
        A.append(a)
        mags.append(mag)
    assert min(mags) >= 0.8 * 2 ** 24 and max(mags) <= 2 ** 24, [m / 2 ** 24 for m in mags]
    n, B = 3 * N - 17, 40
    K = (n + N - 1) // N
    pt = cu(np.full((K, L, d, N), V, dtype=np.uint64))
    db = S.sanns_db_import(ctx, n, pt, cu(np.zeros(K * N, dtype=np.uint32)))
    S.sanns_db_prepare_batched(ctx, db)
    ct_h = np.empty((B, d, 2, L, N), dtype=np.uint64)
    for j in range(L):
        ct_h[:, :, :, j, :] = np.uint64(A[j])
    ct = cu(ct_h)
    acc = S.sanns_distances_batched_mac(ctx, db, ct)
    S.sanns_device_status(ctx)
    acc_plain = S.sanns_distances_mac(ctx, db, ct)
    got = acc.cpu().numpy()
    for j in range(L):
        want = d * A[j] * V % int(qs[j])
        assert np.all(got[:, :, :, j, :] == np.uint64(want)), j
    assert torch.equal(acc.cpu(), acc_plain.cpu())


def test_batched_c3_shape_equals_oracle():
    """The batched configuration's shape (N = 8192, three 60-bit primes,
    d = 96, 64 queries = four 16-query tiles) over three blocks with a ragged
    tail, Gaussian-mixture data: eight of the queries, two per query tile,
    are encrypted by the oracle and their batched responses and server shares
    are compared with the oracle's element by element; all 64 with the
    per-query path."""
    N, L, bits, d, B = 8192, 3, 60, 96, 64
    n = 2 * N + 1000
    ctx = S.sanns_ctx_create(N, L, bits, 0, d)
    coords = inputs.mixture_coords(n, d, 256, 12.0, 31)
    perm = inputs.permutation(n, 32)
    q = inputs.mixture_coords(B, d, 256, 12.0, 33, means_seed=31)
    qids_h = np.arange(100, 100 + B, dtype=np.uint64)
    qids = cu(qids_h)
    sk = S.sanns_keygen(ctx, 34)
    db = S.sanns_encode_db(ctx, cu(coords), cu(perm))
    S.sanns_db_prepare_batched(ctx, db)
    ct = S.sanns_encrypt_query(ctx, sk, cu(q), 35, qids)
    O = Oracle(N, L, bits, 0, d)
    s, s_hat = O.keygen(34)
    picked = [0, 15, 16, 31, 32, 47, 48, 63]
    want_ct = {b: O.encrypt(s_hat, q[b], 35, int(qids_h[b])) for b in picked}
    for b in picked:                       # the oracle's ciphertexts go in
        ct[b] = cu(want_ct[b])
    pt, norms = O.encode_db(coords, perm)
    want = {b: O.intt_mask(O.mac(want_ct[b], pt), norms, n, 0, db.K, 9, int(qids_h[b])) for b in picked}
    po, ps = S.sanns_distances(ctx, db, ct, 9, qids)
    for tile in TILES:
        S.sanns_batched_tune(ctx, tile=tile)
        out, srv = S.sanns_distances_batched(ctx, db, ct, 9, qids)
        S.sanns_device_status(ctx)
        out_h, srv_h = out.cpu().numpy(), srv.cpu().numpy()
        for b in picked:
            assert np.array_equal(out_h[b], want[b][0]), (tile, b)
            assert np.array_equal(srv_h[b], want[b][1]), (tile, b)
        assert torch.equal(po, out) and torch.equal(ps, srv), tile


def test_measured_butterfly_rates_are_plausible():
    """The integer-pipe probe: register-resident butterflies per second are
    positive and below what 148 SMs could issue at one butterfly per lane and
    clock (an upper bound far above any real 64-bit modular butterfly)."""
    ctx = S.sanns_ctx_create(8192, 3, 60, 0, 8)
    r = S.sanns_measure_int_rates(ctx)
    for k in ("inv_butterflies_per_s", "fwd_butterflies_per_s"):
        assert 0 < r[k] < 148 * 128 * 2.1e9, (k, r[k])
