"""GPU parity of the clustering-protocol gather path (one persistent launch
over uneven per-query cluster gathers) against the oracle, which treats each
query's gathered list as a permuted database; also with circuit privacy and
with slot encoding."""
import numpy as np
import pytest
import torch

from oracle.bfv import Oracle
from paper_1904_02033_b300 import inputs
from paper_1904_02033_b300 import sanns as S

pytestmark = pytest.mark.gpu


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gathered_list(offsets, members, probes_b):
    return np.concatenate([members[offsets[c]:offsets[c + 1]] for c in probes_b]
                          + [np.zeros(0, dtype=np.uint32)]).astype(np.uint32)


@pytest.mark.parametrize("cfg,n,C,B,P,F,slots,ntt", [
    ((256, 2, 40, 0, 5), 3000, 20, 3, 4, 0, False, False),
    ((64, 2, 50, 0, 3), 500, 7, 2, 7, 0, False, False),       # probes covering every cluster, tiny N
    ((8192, 3, 60, 0, 4), 30000, 9, 2, 3, 0, False, False),   # N = 8192, three 60-bit primes
    ((256, 3, 60, 0, 5), 3000, 20, 3, 4, 100, False, False),  # circuit privacy
    ((256, 2, 40, 0, 5), 3000, 20, 3, 4, 0, True, False),     # slot encoding
    ((8192, 3, 60, 0, 4), 30000, 9, 2, 3, 148, True, False),  # both, N = 8192
    ((256, 2, 40, 0, 5), 3000, 20, 3, 4, 0, False, True),     # NTT-form responses
    ((256, 3, 60, 0, 5), 3000, 20, 3, 4, 100, True, True),    # all three
    ((8192, 3, 60, 0, 4), 30000, 9, 2, 3, 148, False, True),  # NTT form and privacy, N = 8192
])
def test_gather_matches_oracle(cfg, n, C, B, P, F, slots, ntt):
    N, L, bits, rule, d = cfg
    rnd = np.random.default_rng(n)
    coords = inputs.uniform_coords(n, d, 1)
    # skewed cluster sizes, one empty cluster
    w = inputs.zipf_weights(C, 1.1)
    assign = rnd.choice(C, size=n, p=w)
    assign[assign == C - 1] = 0
    offsets, members = inputs.clusters_csr(assign, C)
    assert offsets[C] - offsets[C - 1] == 0
    probes = np.stack([rnd.permutation(C)[:P] for _ in range(B)]).astype(np.uint32)
    probes[0, -1] = C - 1  # an empty cluster among the probes
    q = inputs.uniform_coords(B, d, 2)
    qids = np.array([5 + 3 * b for b in range(B)], dtype=np.uint64)

    ctx = S.sanns_ctx_create(*cfg)
    sk = S.sanns_keygen(ctx, 3)
    S.sanns_set_encoding(ctx, slots)
    S.sanns_set_response_form(ctx, ntt)
    pk = None
    if F:
        pk_d = S.sanns_public_key(ctx, sk, 8)
        S.sanns_set_circuit_privacy(ctx, pk_d, F)
        pk = pk_d.cpu().numpy()
    cl = S.sanns_clusters_create(ctx, cu(coords), offsets, cu(members))
    ct_in = S.sanns_encrypt_query(ctx, sk, cu(q), 4, cu(qids))
    ct_out, srv, ids, n_b, k_b = S.sanns_distances_gather(ctx, cl, ct_in, probes, 6, cu(qids))
    torch.cuda.synchronize()
    ct_out, srv, ids = ct_out.cpu().numpy(), srv.cpu().numpy(), ids.cpu().numpy()
    ct_np = ct_in.cpu().numpy()

    O = Oracle(*cfg)
    s, _ = O.keygen(3)
    kb0 = nb0 = 0
    for b in range(B):
        g = gathered_list(offsets, members, probes[b])
        assert int(n_b[b]) == len(g) and int(k_b[b]) == -(-len(g) // N)
        assert np.array_equal(ids[nb0:nb0 + len(g)], g)
        if len(g):
            want_out, want_srv = O.distances(ct_np[b], coords, g, 6, int(qids[b]), pk=pk, flood_bits=F,
                                             slots=slots)
            assert np.array_equal(ct_out[kb0:kb0 + int(k_b[b])], O.to_ntt_form(want_out) if ntt else want_out)
            assert np.array_equal(srv[nb0:nb0 + len(g)], want_srv)
            cli = O.decrypt_shares(want_out, s, q[b], len(g), slots=slots)
            brute = np.sum((coords[g].astype(np.int64) - q[b].astype(np.int64)) ** 2, axis=1)
            assert np.array_equal((cli.astype(np.int64) + want_srv) % O.t, brute)
        kb0 += int(k_b[b])
        nb0 += len(g)


def test_gather_rejects_bad_probe():
    ctx = S.sanns_ctx_create(256, 2, 40, 0, 5)
    coords = inputs.uniform_coords(100, 5, 1)
    offsets, members = inputs.clusters_csr(np.arange(100) % 4, 4)
    cl = S.sanns_clusters_create(ctx, cu(coords), offsets, cu(members))
    with pytest.raises(S.SannsError):
        S.sanns_gather_plan(cl, np.array([[0, 4]], dtype=np.uint32))


def _capture(fn):
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        fn()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    return g


@pytest.mark.parametrize("cfg,n,C,B,P,slots", [
    ((256, 2, 40, 0, 5), 3000, 20, 3, 4, False),
    ((8192, 3, 60, 0, 4), 30000, 9, 2, 3, False),
    ((256, 2, 40, 0, 5), 3000, 20, 3, 4, True),
])
def test_prepared_gather_equals_one_shot_and_replays_in_a_graph(cfg, n, C, B, P, slots):
    # the plan uploaded once: eager calls equal the one-shot gather, and the
    # call captured into a CUDA graph and replayed with another batch of
    # ciphertexts in the same buffer equals the one-shot gather of that batch
    N, L, bits, rule, d = cfg
    rnd = np.random.default_rng(n + 1)
    coords = inputs.uniform_coords(n, d, 11)
    assign = rnd.choice(C, size=n, p=inputs.zipf_weights(C, 1.1))
    offsets, members = inputs.clusters_csr(assign, C)
    probes = np.stack([rnd.permutation(C)[:P] for _ in range(B)]).astype(np.uint32)
    qids = cu(np.arange(9, 9 + B, dtype=np.uint64))
    ctx = S.sanns_ctx_create(*cfg)
    sk = S.sanns_keygen(ctx, 12)
    S.sanns_set_encoding(ctx, slots)
    cl = S.sanns_clusters_create(ctx, cu(coords), offsets, cu(members))
    ct_a = S.sanns_encrypt_query(ctx, sk, cu(inputs.uniform_coords(B, d, 13)), 14, qids)
    ct_b = S.sanns_encrypt_query(ctx, sk, cu(inputs.uniform_coords(B, d, 15)), 16, qids)
    ref_a = S.sanns_distances_gather(ctx, cl, ct_a, probes, 6, qids)
    ref_b = S.sanns_distances_gather(ctx, cl, ct_b, probes, 6, qids)
    batch = S.sanns_gather_prepare(ctx, cl, probes)
    assert np.array_equal(batch.n_b, ref_a[3]) and np.array_equal(batch.k_b, ref_a[4])
    tk, tn = int(batch.k_b.sum()), int(batch.n_b.sum())
    ct_in = ct_a.clone()
    out = torch.empty((max(tk, 1), 2, L, N), dtype=torch.uint64, device="cuda")
    srv = torch.empty(max(tn, 1), dtype=torch.uint32, device="cuda")
    ids = torch.empty(max(tn, 1), dtype=torch.uint32, device="cuda")
    S.sanns_distances_gather_prepared(ctx, batch, ct_in, 6, qids, out, srv, ids)
    torch.cuda.synchronize()
    assert torch.equal(out[:tk], ref_a[0]) and torch.equal(srv[:tn], ref_a[1])
    assert torch.equal(ids[:tn], ref_a[2])
    g = _capture(lambda: S.sanns_distances_gather_prepared(ctx, batch, ct_in, 6, qids, out, srv, ids))
    for ct, ref in ((ct_b, ref_b), (ct_a, ref_a)):
        ct_in.copy_(ct)
        out.zero_()
        srv.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out[:tk], ref[0]) and torch.equal(srv[:tn], ref[1])


def test_prepare_rejects_a_probe_past_the_clusters():
    ctx = S.sanns_ctx_create(256, 2, 40, 0, 5)
    offsets, members = inputs.clusters_csr(np.zeros(10, dtype=np.int64), 2)
    cl = S.sanns_clusters_create(ctx, cu(inputs.uniform_coords(10, 5, 1)), offsets, cu(members))
    with pytest.raises(S.SannsError) as e:
        S.sanns_gather_prepare(ctx, cl, np.array([[0, 2]], dtype=np.uint32))
    assert e.value.code == -1
