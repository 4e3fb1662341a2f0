"""Modulus-switched responses (an option beyond the paper, whose server sends
the responses at the full modulus): the GPU's RNS switch equals the oracle's
round(q_0 c / Q) mod q_0 of each coefficient's CRT integer, element by
element, on the per-query, tensor-core and gather paths, with circuit
privacy and slot encoding; decryption modulo q_0 gives the oracle's client
shares, which reconstruct the brute-force distances."""
import numpy as np
import pytest
import torch

from oracle.bfv import Oracle
from paper_1904_02033_b300 import inputs
from paper_1904_02033_b300 import sanns as S

pytestmark = pytest.mark.gpu

_ORACLES = {}


def oracle(*cfg):
    if cfg not in _ORACLES:
        _ORACLES[cfg] = Oracle(*cfg)
    return _ORACLES[cfg]


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _run(cfg, n, B, batched=False, flood=False, slots=False, seed=1):
    N, L, bits, rule, d = cfg
    O = oracle(*cfg)
    coords = inputs.uniform_coords(n, d, seed)
    coords[: min(n, 7)] = 255                      # the largest distances
    perm = inputs.permutation(n, seed + 1)
    q = inputs.uniform_coords(B, d, seed + 2)
    q[0] = 0
    qids = np.arange(20, 20 + B, dtype=np.uint64)
    ctx = S.sanns_ctx_create(*cfg)
    S.sanns_set_encoding(ctx, slots)
    sk = S.sanns_keygen(ctx, seed + 3)
    pk = None
    if flood:
        pk_d = S.sanns_public_key(ctx, sk, seed + 4)
        F = S.sanns_circuit_privacy_max_flood_bits(ctx)
        S.sanns_set_circuit_privacy(ctx, pk_d, F)
        pk = pk_d.cpu().numpy()
    db = S.sanns_encode_db(ctx, cu(coords), cu(perm))
    ct_in = S.sanns_encrypt_query(ctx, sk, cu(q), seed + 5, cu(qids))
    S.sanns_set_response_primes(ctx, 1)
    if batched:
        S.sanns_db_prepare_batched(ctx, db)
        out, srv = S.sanns_distances_batched(ctx, db, ct_in, seed + 6, cu(qids))
    else:
        out, srv = S.sanns_distances(ctx, db, ct_in, seed + 6, cu(qids))
    sw = S.sanns_copy_responses(ctx, out)
    cli = S.sanns_decrypt_shares(ctx, sk, sw, n, cu(q))
    S.sanns_device_status(ctx)
    assert tuple(sw.shape) == (B, db.K, 2, 1, N)
    s_, _ = O.keygen(seed + 3)
    ct_np, sw_np, srv_np, cli_np = (x.cpu().numpy() for x in (ct_in, sw, srv, cli))
    for b in range(B):
        full, srv0 = O.distances(ct_np[b], coords, perm, seed + 6, int(qids[b]), pk=pk,
                                 flood_bits=F if flood else 0, slots=slots)
        want = O.mod_switch(full)
        assert np.array_equal(sw_np[b, :, :, 0], want), b
        assert np.array_equal(srv_np[b], srv0), b
        assert np.array_equal(cli_np[b], O.decrypt_shares_switched(want, s_, q[b], n, slots=slots)), b
        brute = np.sum((coords[perm].astype(np.int64) - q[b].astype(np.int64)) ** 2, axis=1)
        assert np.array_equal((cli_np[b].astype(np.int64) + srv_np[b]) % O.t, brute), b
    return ctx, sk, out, sw, cli, q


@pytest.mark.parametrize("cfg,n,B", [
    ((256, 2, 40, 0, 5), 600, 2),            # one dropped prime, three blocks, ragged
    ((256, 3, 60, 1, 17), 700, 1),           # two dropped primes, t = 2^b_d
    ((64, 4, 60, 0, 3), 64 * 3 - 1, 2),      # three dropped primes (Garner over three digits)
    ((8192, 3, 60, 0, 7), 8192 * 2 + 5, 1),  # N = 8192, three 60-bit primes
])
def test_switched_responses_equal_oracle(cfg, n, B):
    _run(cfg, n, B)


def test_switched_responses_on_the_tensor_core_path():
    _run((256, 3, 60, 0, 16), 256 * 40 - 9, 3, batched=True, seed=4)


@pytest.mark.parametrize("cfg", [(256, 2, 40, 0, 5), (256, 3, 60, 0, 8)])
def test_switched_responses_with_maximum_flooding(cfg):
    _run(cfg, 2 * cfg[0] - 3, 2, flood=True, seed=7)


def test_switched_responses_with_slot_encoding():
    _run((256, 2, 40, 0, 5), 700, 2, slots=True, seed=9)


def test_copies_and_noalloc_decryption_agree():
    ctx, sk, out, sw, cli, q = _run((256, 3, 60, 0, 6), 500, 2, seed=11)
    host = torch.empty(tuple(sw.shape), dtype=torch.uint64).pin_memory()
    S.sanns_copy_responses(ctx, out, host)
    torch.cuda.synchronize()
    assert torch.equal(host, sw.cpu())
    # the switched rows are row 0 of each response in the distance buffer
    assert torch.equal(out[:, :, :, 0:1].contiguous().cpu(), sw.cpu())
    cli2 = S.sanns_decrypt_shares_noalloc(ctx, sk, sw, 500, q=cu(q))
    torch.cuda.synchronize()
    assert torch.equal(cli2.cpu(), cli.cpu())
    # at every prime the copy is the whole response buffer
    S.sanns_set_response_primes(ctx, 3)
    full = S.sanns_copy_responses(ctx, out)
    torch.cuda.synchronize()
    assert tuple(full.shape) == tuple(out.shape) and torch.equal(full, out)


def test_switching_rules():
    ctx = S.sanns_ctx_create(256, 3, 60, 0, 5)
    with pytest.raises(S.SannsError):
        S.sanns_set_response_primes(ctx, 2)            # 1 or L only
    S.sanns_set_response_form(ctx, True)
    with pytest.raises(S.SannsError):
        S.sanns_set_response_primes(ctx, 1)            # NTT form cannot be switched
    S.sanns_set_response_form(ctx, False)
    S.sanns_set_response_primes(ctx, 1)
    with pytest.raises(S.SannsError):
        S.sanns_set_response_form(ctx, True)


@pytest.mark.parametrize("cfg,F", [((256, 3, 60, 0, 5), 0), ((256, 2, 40, 0, 5), 30)])
def test_switched_gather_responses_equal_oracle(cfg, F):
    # the clustering gather switches each work item's response the same way
    N, L, bits, rule, d = cfg
    n, C, B, P = 3000, 20, 3, 4
    rnd = np.random.default_rng(n + L)
    coords = inputs.uniform_coords(n, d, 1)
    assign = rnd.choice(C, size=n, p=inputs.zipf_weights(C, 1.1))
    offsets, members = inputs.clusters_csr(assign, C)
    probes = np.stack([rnd.permutation(C)[:P] for _ in range(B)]).astype(np.uint32)
    q = inputs.uniform_coords(B, d, 2)
    qids = np.array([5 + 3 * b for b in range(B)], dtype=np.uint64)
    ctx = S.sanns_ctx_create(*cfg)
    sk = S.sanns_keygen(ctx, 3)
    pk = None
    if F:
        pk_d = S.sanns_public_key(ctx, sk, 8)
        S.sanns_set_circuit_privacy(ctx, pk_d, F)
        pk = pk_d.cpu().numpy()
    S.sanns_set_response_primes(ctx, 1)
    cl = S.sanns_clusters_create(ctx, cu(coords), offsets, cu(members))
    ct_in = S.sanns_encrypt_query(ctx, sk, cu(q), 4, cu(qids))
    ct_out, srv, ids, n_b, k_b = S.sanns_distances_gather(ctx, cl, ct_in, probes, 6, cu(qids))
    W = int(k_b.sum())
    sw = S.sanns_copy_responses(ctx, ct_out[:W].reshape(1, W, 2, L, N)).reshape(W, 2, N)
    S.sanns_device_status(ctx)
    sw, srv, ct_np = sw.cpu().numpy(), srv.cpu().numpy(), ct_in.cpu().numpy()
    O = oracle(*cfg)
    s_, _ = O.keygen(3)
    kb0 = nb0 = 0
    for b in range(B):
        g = np.concatenate([members[offsets[c]:offsets[c + 1]] for c in probes[b]]).astype(np.uint32)
        full, want_srv = O.distances(ct_np[b], coords, g, 6, int(qids[b]), pk=pk, flood_bits=F)
        want = O.mod_switch(full)
        assert np.array_equal(sw[kb0:kb0 + int(k_b[b])], want), b
        assert np.array_equal(srv[nb0:nb0 + len(g)], want_srv), b
        cli = O.decrypt_shares_switched(want, s_, q[b], len(g))
        brute = np.sum((coords[g].astype(np.int64) - q[b].astype(np.int64)) ** 2, axis=1)
        assert np.array_equal((cli.astype(np.int64) + want_srv) % O.t, brute), b
        kb0 += int(k_b[b])
        nb0 += len(g)
