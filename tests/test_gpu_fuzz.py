"""Seeded random configurations through the whole per-query step, each
against the oracle: ring size, prime count and size, dimension, database
size (ragged), queries per call, MAC launch variant and response form
(full modulus or switched down to q_0) are drawn from a fixed stream, so the
epilogue kernels chosen by launch size (the cluster, short and fused
INTT + mask kernels) and every MAC variant meet shapes the hand-written
cases do not."""
import numpy as np
import pytest
import torch

from oracle.bfv import Oracle
from paper_1904_02033_b300 import inputs
from paper_1904_02033_b300 import sanns as S

pytestmark = pytest.mark.gpu

CASES = 40


def _case(i):
    rnd = np.random.default_rng(1000 + i)
    N = int(rnd.choice([256, 1024, 2048, 4096]))
    L = int(rnd.integers(2, 5))
    bits = int(rnd.choice([50, 55, 60]))
    d = int(rnd.integers(1, 41))
    n = int(rnd.integers(1, 6 * N + 1))
    B = int(rnd.integers(1, 7))
    switched = bool(rnd.random() < 0.4)
    return (N, L, bits, 0, d), n, B, switched, int(rnd.integers(0, 1 << 30))


@pytest.mark.parametrize("i", range(CASES))
def test_random_configuration_matches_oracle(i):
    cfg, n, B, switched, seed = _case(i)
    N, L, bits, rule, d = cfg
    ctx = S.sanns_ctx_create(*cfg)
    variant = seed % len(S.sanns_mac_variants())
    S.sanns_set_mac_variant(ctx, variant)
    coords = inputs.uniform_coords(n, d, seed)
    coords[: min(n, 3)] = 255
    perm = inputs.permutation(n, seed + 1)
    q = inputs.uniform_coords(B, d, seed + 2)
    qids = np.arange(7, 7 + B, dtype=np.uint64) * 1009
    sk = S.sanns_keygen(ctx, seed + 3)
    db = S.sanns_encode_db(ctx, torch.from_numpy(coords).cuda(), torch.from_numpy(perm).cuda())
    ct_in = S.sanns_encrypt_query(ctx, sk, torch.from_numpy(q).cuda(), seed + 4,
                                  torch.from_numpy(qids).cuda())
    if switched:
        S.sanns_set_response_primes(ctx, 1)
    out, srv = S.sanns_distances(ctx, db, ct_in, seed + 5, torch.from_numpy(qids).cuda())
    resp = S.sanns_copy_responses(ctx, out) if switched else out
    cli = S.sanns_decrypt_shares(ctx, sk, resp, n, torch.from_numpy(q).cuda())
    S.sanns_device_status(ctx)
    O = Oracle(*cfg)
    s_, _ = O.keygen(seed + 3)
    ct_np, resp_np, srv_np, cli_np = (x.cpu().numpy() for x in (ct_in, resp, srv, cli))
    name = (cfg, n, B, switched, S.sanns_mac_variants()[variant])
    for b in range(B):
        full, want_srv = O.distances(ct_np[b], coords, perm, seed + 5, int(qids[b]))
        assert np.array_equal(srv_np[b], want_srv), (name, b)
        if switched:
            want = O.mod_switch(full)
            assert np.array_equal(resp_np[b, :, :, 0], want), (name, b)
            want_cli = O.decrypt_shares_switched(want, s_, q[b], n)
        else:
            assert np.array_equal(resp_np[b], full), (name, b)
            want_cli = O.decrypt_shares(full, s_, q[b], n)
        assert np.array_equal(cli_np[b], want_cli), (name, b)
        brute = np.sum((coords[perm].astype(np.int64) - q[b].astype(np.int64)) ** 2, axis=1)
        assert np.array_equal((cli_np[b].astype(np.int64) + srv_np[b]) % O.t, brute), (name, b)


@pytest.mark.parametrize("i", range(16))
def test_random_batched_configuration_equals_per_query_and_oracle(i):
    """The tensor-core path on seeded random shapes (ring, primes, d up to
    the exactness limit 128, ragged database, 1..40 queries, tile shape,
    scratch cap): every query equals the per-query path, and the first
    query's blocks equal the oracle."""
    rnd = np.random.default_rng(5000 + i)
    N = int(rnd.choice([256, 512, 1024]))
    L = int(rnd.integers(2, 5))
    cfg = (N, L, int(rnd.choice([50, 60])), 0, int(rnd.integers(1, 129)))
    d = cfg[4]
    n = int(rnd.integers(1, 300 * 256 + 1))   # up to 300 blocks at N = 256 (several database tiles)
    B = int(rnd.integers(1, 41))
    tile = int(rnd.integers(0, 9))
    scratch = int(rnd.choice([2, 8, 4096]))
    seed = int(rnd.integers(0, 1 << 30))
    ctx = S.sanns_ctx_create(*cfg)
    coords = inputs.uniform_coords(n, d, seed)
    perm = inputs.permutation(n, seed + 1)
    q = inputs.uniform_coords(B, d, seed + 2)
    qids = np.arange(B, dtype=np.uint64) * 31 + 5
    sk = S.sanns_keygen(ctx, seed + 3)
    db = S.sanns_encode_db(ctx, torch.from_numpy(coords).cuda(), torch.from_numpy(perm).cuda())
    S.sanns_db_prepare_batched(ctx, db)
    ct_in = S.sanns_encrypt_query(ctx, sk, torch.from_numpy(q).cuda(), seed + 4,
                                  torch.from_numpy(qids).cuda())
    S.sanns_batched_tune(ctx, scratch_mib=scratch, tile=tile)
    qd = torch.from_numpy(qids).cuda()
    out_b, srv_b = S.sanns_distances_batched(ctx, db, ct_in, seed + 5, qd)
    S.sanns_device_status(ctx)
    out_p, srv_p = S.sanns_distances(ctx, db, ct_in, seed + 5, qd)
    name = (cfg, n, B, tile, scratch)
    assert torch.equal(out_b, out_p) and torch.equal(srv_b, srv_p), name
    O = Oracle(*cfg)
    full, want_srv = O.distances(ct_in[0].cpu().numpy(), coords, perm, seed + 5, int(qids[0]))
    assert np.array_equal(out_b[0].cpu().numpy(), full), name
    assert np.array_equal(srv_b[0].cpu().numpy(), want_srv), name


def _gathered(offsets, members, probes):
    parts = [members[offsets[c]:offsets[c + 1]] for c in probes]
    return np.concatenate(parts).astype(np.uint32) if parts else np.zeros(0, np.uint32)


@pytest.mark.parametrize("i", range(16))
def test_random_gather_matches_oracle(i):
    """The clustering gather on seeded random clusterings: ring, primes,
    dimension, skewed cluster sizes (some empty), queries and probes per
    query, with slot encoding, NTT-form or switched responses and circuit
    privacy drawn at random; each query's responses and shares equal the
    oracle's linear scan of its gathered list."""
    rnd = np.random.default_rng(9000 + i)
    N = int(rnd.choice([256, 1024, 4096]))
    L = int(rnd.integers(2, 4))
    cfg = (N, L, 60, 0, int(rnd.integers(1, 33)))
    d = cfg[4]
    n = int(rnd.integers(50, 4 * N + 1))
    C = int(rnd.integers(2, 40))
    B = int(rnd.integers(1, 7))
    P = int(rnd.integers(1, C + 1))
    slots = bool(rnd.random() < 0.25)
    ntt = bool(rnd.random() < 0.25)
    switched = (not ntt) and bool(rnd.random() < 0.3)
    F = int(rnd.choice([0, 0, 0, 60]))
    seed = int(rnd.integers(0, 1 << 30))
    coords = inputs.uniform_coords(n, d, seed)
    assign = rnd.choice(C, size=n, p=inputs.zipf_weights(C, 1.1))
    offsets, members = inputs.clusters_csr(assign, C)
    probes = np.stack([rnd.permutation(C)[:P] for _ in range(B)]).astype(np.uint32)
    q = inputs.uniform_coords(B, d, seed + 1)
    qids = np.arange(B, dtype=np.uint64) * 7 + 3
    ctx = S.sanns_ctx_create(*cfg)
    sk = S.sanns_keygen(ctx, seed + 2)
    S.sanns_set_encoding(ctx, slots)
    S.sanns_set_response_form(ctx, ntt)
    pk = None
    if F:
        pk_d = S.sanns_public_key(ctx, sk, seed + 3)
        S.sanns_set_circuit_privacy(ctx, pk_d, F)
        pk = pk_d.cpu().numpy()
    if switched:
        S.sanns_set_response_primes(ctx, 1)
    cl = S.sanns_clusters_create(ctx, torch.from_numpy(coords).cuda(), offsets,
                                 torch.from_numpy(members).cuda())
    ct_in = S.sanns_encrypt_query(ctx, sk, torch.from_numpy(q).cuda(), seed + 4,
                                  torch.from_numpy(qids).cuda())
    ct_out, srv, ids, n_b, k_b = S.sanns_distances_gather(ctx, cl, ct_in, probes, seed + 5,
                                                          torch.from_numpy(qids).cuda())
    S.sanns_device_status(ctx)
    W = int(k_b.sum())
    if switched and W:
        ct_out = S.sanns_copy_responses(ctx, ct_out[:W].reshape(1, W, 2, L, N)).reshape(W, 2, N)
    ct_out, srv, ids, ct_np = ct_out.cpu().numpy(), srv.cpu().numpy(), ids.cpu().numpy(), ct_in.cpu().numpy()
    O = Oracle(*cfg)
    name = (cfg, n, C, B, P, slots, ntt, switched, F)
    kb0 = nb0 = 0
    for b in range(B):
        g = _gathered(offsets, members, probes[b])
        assert int(n_b[b]) == len(g) and int(k_b[b]) == -(-len(g) // N), name
        assert np.array_equal(ids[nb0:nb0 + len(g)], g), name
        if len(g):
            want, want_srv = O.distances(ct_np[b], coords, g, seed + 5, int(qids[b]), pk=pk, flood_bits=F,
                                         slots=slots)
            if ntt:
                want = O.to_ntt_form(want)
            elif switched:
                want = O.mod_switch(want)
            assert np.array_equal(ct_out[kb0:kb0 + int(k_b[b])], want), (name, b)
            assert np.array_equal(srv[nb0:nb0 + len(g)], want_srv), (name, b)
        kb0 += int(k_b[b])
        nb0 += len(g)
