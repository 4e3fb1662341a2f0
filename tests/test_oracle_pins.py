"""Pins for the CPU oracle: each test checks the oracle against something other
than itself -- a definition evaluated independently, a library routine, a
published test vector or value, or an identity the method must satisfy.
"""
import math
import os
import random

import numpy as np
import pytest
import sympy

from oracle import chacha20_block
from oracle.bfv import Oracle
from oracle.params import make_params, ntt_primes, plain_modulus, min_primitive_root_2n
from oracle import select
from paper_1904_02033_b300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- params
@pytest.mark.parametrize("N,L,bits", [(4096, 2, 54), (8192, 3, 60), (256, 2, 40), (64, 3, 30)])
def test_primes_are_the_largest_ntt_primes(N, L, bits):
    qs = ntt_primes(N, L, bits)
    assert qs == sorted(qs, reverse=True) and len(set(qs)) == L
    for q in qs:
        assert sympy.isprime(q) and q % (2 * N) == 1 and q < 2 ** bits
    # nothing skipped: every candidate = 1 mod 2N between q_L and 2^bits
    # that is not in the list is composite (sympy decides)
    x = qs[-1]
    while x < 2 ** bits:
        if x not in qs:
            assert not sympy.isprime(x)
        x += 2 * N


def test_ntt_primes_match_printed_modulus_size():
    # Sec. 7.1: N = 2^13 and a 180-bit modulus q made of three RNS words
    P = make_params(8192, 3, 60, 0, 128)
    assert P.Q.bit_length() == 180


@pytest.mark.parametrize("N,bits", [(8, 20), (16, 30), (64, 40), (256, 54)])
def test_psi_is_the_smallest_primitive_root(N, bits):
    q = ntt_primes(N, 1, bits)[0]
    psi = min_primitive_root_2n(q, N)
    assert pow(psi, N, q) == q - 1
    if N <= 16:
        # brute force over all residues for tiny q is too big; instead compare
        # with sympy's full list of N-th roots of -1
        roots = sympy.nthroot_mod(q - 1, N, q, all_roots=True)
        assert psi == min(roots)


def test_plain_modulus_paper_rule_matches_printed_t():
    # Sec. 7.1 prints t = 2^23 (SIFT, Deep1B) and t = 2^24 (Amazon); the rule
    # b_d = 2 b_c + ceil(log2 d) comes from Fig. "hyperparameters".
    rows = [l.split() for l in open(os.path.join(GOLD, "paper_comm_bytes.txt"))
            if l.strip() and not l.startswith("#")]
    trows = [r for r in rows if len(r) == 4 and r[1] in ("8", "9")]
    assert len(trows) == 3
    for name, b_c, d, t in trows:
        assert plain_modulus(8192, 1, int(d), int(b_c)) == int(t), name


def test_plain_modulus_prime_rule():
    for N in (4096, 8192):
        t = plain_modulus(N, 0, 128)
        assert sympy.isprime(t) and t % (2 * N) == 1 and t > 2 ** 24
        x = 2 ** 24 + 1
        while x < t:
            if x % (2 * N) == 1:
                assert not sympy.isprime(x)
            x += 1 if x % (2 * N) != 1 else 2 * N
    # every squared distance of 8-bit points fits below t, so the shares
    # reconstruct the exact integer (Sec. 5.3)
    assert 128 * 255 ** 2 < plain_modulus(8192, 0, 128)


def test_ciphertext_layout_reproduces_paper_communication():
    # d query ciphertexts + ceil(n/N) response ciphertexts, each 2 polys x
    # 3 RNS words x N coefficients x 8 bytes, equals the printed MB figures.
    rows = [l.split() for l in open(os.path.join(GOLD, "paper_comm_bytes.txt"))
            if l.strip() and not l.startswith("#")]
    crow = [r for r in rows if len(r) == 4 and "." in r[3] or r[3] == "518"]
    assert len(crow) == 4
    N, L = 8192, 3
    for name, n, d, mb in crow:
        n, d = int(n), int(d)
        K = -(-n // N)
        ct_in = d * 2 * L * N * 8
        ct_out = K * 2 * L * N * 8
        got = (ct_in + ct_out) / 1e6
        digits = len(mb.replace(".", "").lstrip("0"))
        assert float(f"{got:.{digits}g}") == float(mb), (name, got, mb)


# ---------------------------------------------------------------- ChaCha20
def test_chacha20_rfc8439_block_vector():
    kv = {}
    for line in open(os.path.join(GOLD, "chacha20_rfc8439.txt")):
        if line.strip() and not line.startswith("#"):
            k, *v = line.split()
            kv[k] = v
    key = [int(w, 16) for w in kv["key_words"]]
    nonce = [int(w, 16) for w in kv["nonce_words"]]
    out = chacha20_block(key, int(kv["counter"][0]), nonce)
    assert out.astype("<u4").tobytes().hex() == kv["block"][0]



def test_draw128_layout_over_the_rfc_block():
    # The 128-bit draw of coefficient c of stream (seed, purpose, object):
    # key = seed as two little-endian words, nonce = (purpose, object low,
    # object high), block counter c / 4, words 4 (c mod 4) .. + 3 of the block.
    # With seed = purpose = object = 0 the eight draws c = 0 .. 7 are the RFC
    # 8439 A.1 zero-key keystream (block counters 0 and 1) read in order.
    g = {}
    for line in open(os.path.join(GOLD, "chacha20_rfc8439_zero_key.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            g[k] = v
    O = Oracle(64, 1, 40, 0, 1)
    stream = bytes.fromhex(g["block0"] + g["block1"])
    for c in range(8):
        lo, hi = O.draw128(0, 0, 0, c)
        assert ((hi << 64) | lo).to_bytes(16, "little") == stream[16 * c:16 * c + 16], c
    rnd = random.Random(7)
    for _ in range(40):
        seed, purpose = rnd.getrandbits(64), rnd.randrange(1, 11)
        obj, c = rnd.getrandbits(40), rnd.getrandbits(33)
        blk = chacha20_block([seed & 0xFFFFFFFF, seed >> 32, 0, 0, 0, 0, 0, 0], c // 4,
                             [purpose, obj & 0xFFFFFFFF, obj >> 32])
        w = [int(x) for x in blk[4 * (c % 4):4 * (c % 4) + 4]]
        assert O.draw128(seed, purpose, obj, c) == (w[0] | w[1] << 32, w[2] | w[3] << 32)


# ---------------------------------------------------------------- NTT
def _ntt_definition(a, q, psi):
    """O(N^2) definition of the convention: slot s holds a(psi^(2 brv(s)+1))."""
    N = len(a)
    logn = N.bit_length() - 1
    out = []
    for s in range(N):
        r = int(format(s, f"0{logn}b")[::-1], 2) if logn else 0
        x = pow(psi, 2 * r + 1, q)
        acc = 0
        for c in reversed(a):
            acc = (acc * x + int(c)) % q
        out.append(acc)
    return out


def _negacyclic(a, b, q):
    N = len(a)
    out = [0] * N
    for i in range(N):
        for j in range(N):
            k = i + j
            p = int(a[i]) * int(b[j])
            if k < N:
                out[k] += p
            else:
                out[k - N] -= p
    return [v % q for v in out]


@pytest.mark.parametrize("N,bits", [(8, 20), (16, 30), (64, 54), (256, 60)])
def test_ntt_matches_definition_and_inverts(N, bits):
    O = Oracle(N, 2, bits, 0, 4)
    rnd = np.random.default_rng(N)
    for j in range(2):
        q = int(O.q[j])
        for case in range(3):
            if case == 0:
                a = rnd.integers(0, q, size=N, dtype=np.uint64)
            elif case == 1:
                a = np.full(N, q - 1, dtype=np.uint64)
            else:
                a = np.zeros(N, dtype=np.uint64)
                a[rnd.integers(0, N)] = rnd.integers(1, q)
            f = O.ntt(a, j)
            assert [int(v) for v in f] == _ntt_definition(a, q, O.P.psi[j])
            assert np.array_equal(O.intt(f, j), a)


@pytest.mark.parametrize("N,bits", [(8, 20), (32, 54), (128, 60)])
def test_ntt_product_is_negacyclic_product(N, bits):
    O = Oracle(N, 1, bits, 0, 4)
    q = int(O.q[0])
    rnd = np.random.default_rng(7)
    a = rnd.integers(0, q, size=N, dtype=np.uint64)
    b = rnd.integers(0, q, size=N, dtype=np.uint64)
    fa, fb = O.ntt(a, 0), O.ntt(b, 0)
    prod = np.array([(int(x) * int(y)) % q for x, y in zip(fa, fb)], dtype=np.uint64)
    got = O.intt(prod, 0)
    want = _negacyclic(a, b, q)
    assert [int(v) for v in got] == want
    assert [int(v) for v in O.schoolbook(a, b, 0)] == want


# ---------------------------------------------------------------- BFV
def _small():
    return Oracle(256, 2, 40, 0, 5)


def test_keygen_is_ternary_and_ntt_of_s():
    O = _small()
    s, s_hat = O.keygen(seed=3)
    assert set(np.unique(s)).issubset({-1, 0, 1})
    counts = np.bincount(s.astype(np.int64) + 1, minlength=3)
    assert counts.min() > 256 / 3 * 0.6
    # the secret's stream: s_x = (lo mod 3) - 1 of the 128-bit draw x of
    # (seed, purpose 1, object 0), read from the RFC-pinned block function
    # with the documented key / nonce / counter / word layout
    for seed in (3, 0xFEDCBA9876543210):
        sx = O.keygen(seed=seed)[0]
        for x in range(O.N):
            blk = chacha20_block([seed & 0xFFFFFFFF, seed >> 32, 0, 0, 0, 0, 0, 0], x // 4, [1, 0, 0])
            lo = int(blk[4 * (x % 4)]) | int(blk[4 * (x % 4) + 1]) << 32
            assert int(sx[x]) == lo % 3 - 1, (seed, x)
    for j in range(O.L):
        q = int(O.q[j])
        lifted = [(int(v) % q) for v in s]
        assert [int(v) for v in s_hat[j]] == _ntt_definition(lifted, q, O.P.psi[j])


def test_decrypt_of_encrypt_is_the_constant_plaintext():
    O = _small()
    s, s_hat = O.keygen(seed=1)
    qv = np.array([0, 1, 7, 128, 255], dtype=np.uint8)
    ct = O.encrypt(s_hat, qv, seed=11, qid=5)
    # back to coefficient form, then decrypt each coordinate's ciphertext
    ctc = np.zeros_like(ct)
    for i in range(O.d):
        for c in range(2):
            for j in range(O.L):
                ctc[i, c, j] = O.intt(ct[i, c, j], j)
    v = O.decrypt_phase(ctc, s)
    m = O.scale_round(v).reshape(O.d, O.N)
    for i in range(O.d):
        want = np.zeros(O.N, dtype=np.int64)
        want[0] = (O.t - 2 * int(qv[i])) % O.t
        assert np.array_equal(m[i], want)
    assert O.noise_ok(v, m.reshape(-1))
    # c1 is not a constant: the ciphertext actually hides the message
    assert len(np.unique(ct[0, 1, 0])) > O.N // 2


def _distances_case(O, n, seed, perm=True, qid=9):
    coords = inputs.uniform_coords(n, O.d, seed)
    qv = inputs.uniform_coords(1, O.d, seed + 1)[0]
    pm = inputs.permutation(n, seed + 2) if perm else None
    s, s_hat = O.keygen(seed=seed + 3)
    ct = O.encrypt(s_hat, qv, seed=seed + 4, qid=qid)
    out, srv = O.distances(ct, coords, pm, mask_seed=seed + 5, qid=qid)
    cli = O.decrypt_shares(out, s, qv, n)
    order = np.arange(n) if pm is None else pm
    brute = np.sum((coords[order].astype(np.int64) - qv.astype(np.int64)) ** 2, axis=1)
    return cli, srv, brute


@pytest.mark.parametrize("n", [1, 255, 256, 600])
def test_shares_reconstruct_bruteforce_distances(n):
    """Sec. 5.3: sum_i f_i g_i holds <q, p_j> in coefficient j; with the
    client's -2 factor, the server's ||p||^2 and the mask the two shares add
    up to ||q - p||^2 mod t, and t exceeds every such distance."""
    O = _small()
    cli, srv, brute = _distances_case(O, n, seed=n)
    assert np.array_equal((cli.astype(np.int64) + srv) % O.t, brute)
    if n > 16:
        # the mask hides the distances: the client share alone is not them
        assert np.mean(cli.astype(np.int64) == brute) < 0.1


def test_shares_at_small_config_scale():
    """N = 4096, two 54-bit primes, d = 32, n = 4096 (one block)."""
    O = Oracle(4096, 2, 54, 0, 32)
    cli, srv, brute = _distances_case(O, 4096, seed=0)
    assert np.array_equal((cli.astype(np.int64) + srv) % O.t, brute)


def test_shares_with_paper_power_of_two_t():
    O = Oracle(256, 3, 60, 1, 5)
    assert O.t == 2 ** 19
    cli, srv, brute = _distances_case(O, 300, seed=4)
    assert np.array_equal((cli.astype(np.int64) + srv) % O.t, brute)


def test_block_ranges_compose():
    O = _small()
    n = 700
    coords = inputs.uniform_coords(n, O.d, 1)
    s, s_hat = O.keygen(seed=2)
    qv = inputs.uniform_coords(1, O.d, 3)[0]
    ct = O.encrypt(s_hat, qv, seed=4, qid=1)
    full, srv = O.distances(ct, coords, None, 5, 1)
    parts = [O.distances(ct, coords, None, 5, 1, k0=k, k1=k + 1) for k in range(3)]
    assert np.array_equal(np.concatenate([p[0] for p in parts]), full)
    assert np.array_equal(np.concatenate([p[1] for p in parts]), srv)


# ---------------------------------------------------------------- selection
def test_naive_topk_is_sorted_selection():
    rnd = random.Random(5)
    for _ in range(20):
        n = rnd.randint(1, 60)
        k = rnd.randint(1, 12)
        vals = [rnd.randint(0, 9) for _ in range(n)]
        ids = list(range(100, 100 + n))
        opt, idl = select.naive_topk(vals, ids, k)
        ev, ei = select.exact_topk(np.array(vals), np.array(ids), k)
        m = min(n, k)
        # the values are unique; under ties Algorithm 1 may order equal
        # values differently, so check the ids form a valid selection
        assert opt[:m] == ev
        assert len(set(idl[:m])) == m
        assert all(vals[i - 100] == v for i, v in zip(idl[:m], opt[:m]))
        if len(set(vals)) == n:
            assert idl[:m] == ei


def test_approx_topk_with_one_bin_per_element_is_exact():
    rnd = np.random.default_rng(1)
    v = rnd.integers(0, 1000, size=200)
    ids = np.arange(200)
    assert select.approx_topk(v, ids, 10, 200) == select.exact_topk(v, ids, 10)


def test_approx_topk_expected_hits_closed_forms():
    # independent-bins model of the Theorem 1 proof: l (1 - (1 - 1/l)^k);
    # with fixed bins the hypergeometric value is close to it for large n
    n, k, l = 10 ** 6, 10, 7813
    indep = l * (1 - (1 - 1 / l) ** k)
    fixed = select.expected_hits(n, k, l)
    assert abs(indep - fixed) < 1e-3
    assert 9.99 < fixed < 10
    # Monte Carlo on a small case
    n, k, l = 2000, 10, 40
    rnd = np.random.default_rng(0)
    v = np.arange(n)
    hits = []
    for _ in range(400):
        pm = rnd.permutation(n)
        vals = v[pm]
        _, got = select.approx_topk(vals, pm, k, l)
        hits.append(len(set(got) & set(range(k))))
    want = select.expected_hits(n, k, l)
    assert abs(np.mean(hits) - want) < 4 * np.std(hits) / math.sqrt(len(hits)) + 0.02



@pytest.mark.parametrize("n,k,l", [(7, 3, 3), (7, 2, 4), (6, 3, 5)])
def test_expected_hits_equals_brute_force_over_all_permutations(n, k, l):
    # E|I| of Algorithm 2 by enumeration: every ordering of n distinct values
    # run through ApproxTopk, the true top k counted among its output
    import itertools
    v = np.arange(n)
    tot, cnt = 0, 0
    for pm in itertools.permutations(range(n)):
        pm = np.array(pm)
        _, got = select.approx_topk(v[pm], pm, k, l)
        tot += len(set(got) & set(range(k)))
        cnt += 1
    assert abs(tot / cnt - select.expected_hits(n, k, l)) < 1e-12


@pytest.mark.parametrize("k", [5, 10, 20, 50, 100])
@pytest.mark.parametrize("delta", [0.01, 0.02, 0.05, 0.1])
def test_theorem_1_bins_k_over_delta_meet_the_bound(k, delta):
    # Theorem 1: with l = k / delta bins the expected number of true top-k
    # entries returned is at least (1 - delta) k; checked on the Sec. 7
    # selection grid (n = 10^6 values, k and delta as evaluated there)
    n = 10 ** 6
    l = math.ceil(k / delta)
    assert select.expected_hits(n, k, l) >= (1 - delta) * k


# ---------------------------------------------------------------------------
# circuit privacy (Sec. 2.3 "Additive Homomorphic Encryption": circuit privacy by
# noise flooding; a public key lets the server re-randomise c1)
# ---------------------------------------------------------------------------
def test_public_key_is_an_encryption_of_zero():
    O = Oracle(256, 2, 60, 0, 3)
    s, s_hat = O.keygen(11)
    pk = O.public_key(s_hat, 12)
    ct = np.zeros((1, 2, O.L, O.N), dtype=np.uint64)
    for c in range(2):
        for j in range(O.L):
            ct[0, c, j] = O.intt(pk[c, j], j)
    v = O.decrypt_phase(ct, s)          # c0 + c1 s = e, the same small integer per prime
    for j in range(O.L):
        q = int(O.q[j])
        cen = [int(x) if int(x) <= q // 2 else int(x) - q for x in v[0, j]]
        assert max(abs(x) for x in cen) <= 21 and any(cen)
        if j:
            assert cen == prev
        prev = cen


@pytest.mark.parametrize("F", [0, 120])
def test_circuit_privacy_keeps_shares_and_floods_the_noise(F):
    cfg = (256, 3, 60, 0, 5)
    O = Oracle(*cfg)
    n, d = 256 * 3 - 7, cfg[4]
    rnd = np.random.default_rng(F + 1)
    coords = rnd.integers(0, 256, size=(n, d), dtype=np.uint8)
    qv = rnd.integers(0, 256, size=d, dtype=np.uint8)
    s, s_hat = O.keygen(21)
    pk = O.public_key(s_hat, 22)
    ct = O.encrypt(s_hat, qv, 23, 5)
    plain, srv0 = O.distances(ct, coords, None, 24, 5)
    priv, srv = O.distances(ct, coords, None, 24, 5, pk=pk, flood_bits=F)
    assert np.array_equal(srv, srv0)                    # the mask is unchanged
    assert not np.array_equal(priv[:, 1], plain[:, 1])  # c1 re-randomised
    cli = O.decrypt_shares(priv, s, qv, n)
    brute = np.sum((coords.astype(np.int64) - qv.astype(np.int64)) ** 2, axis=1)
    assert np.array_equal((cli.astype(np.int64) + srv) % O.t, brute)
    # the phase noise is the flooding term: about 2^F, and below Delta / 2
    m = O.scale_round(O.decrypt_phase(priv, s))
    noise = max(O.phase_noise(priv, s, m))
    if F:
        assert 2 ** (F - 2) <= noise <= 2 ** F + 2 ** 50
    else:
        assert noise < 2 ** 50
    assert noise < O.P.delta // 2


@pytest.mark.parametrize("seed", range(6))
def test_approx_topk_by_position_selects_algorithm_2_values(seed):
    rnd = np.random.default_rng(seed)
    n = int(rnd.integers(40, 400))
    vals = rnd.integers(0, 6, size=n)             # many ties
    ids = np.arange(n)
    for l in (10, n // 3, n):
        k = min(10, l)
        lit_v, lit_i = select.approx_topk(vals, ids, k, l)
        pos_v, pos_i = select.approx_topk_by_position(vals, ids, k, l)
        assert pos_v == lit_v                      # the same values in the same order
        b = select.bin_of(n, l)
        mins = {}
        for x in range(n):
            if b[x] not in mins or vals[x] < vals[mins[b[x]]]:
                mins[b[x]] = x
        minpos = set(mins.values())
        assert set(pos_i) <= minpos and set(lit_i) <= minpos   # both pick bin minima
        assert len(set(pos_i)) == k
        assert pos_i == sorted(pos_i, key=lambda x: (vals[x], x))


# ---------------------------------------------------------------- Algorithm 4
def _toy_layout(n, d, C, seed, stash_n=0):
    """A hand-made layout: C clusters of a random assignment (some points kept
    back as the stash), one group per two thirds / one third of the clusters,
    centres = rounded member means in a seeded shuffled order."""
    rnd = np.random.default_rng(seed)
    coords = inputs.mixture_coords(n, d, 6, 25.0, seed)
    order = rnd.permutation(n)
    stash = np.sort(order[:stash_n]).astype(np.int64)
    rest = np.sort(order[stash_n:])
    assign = rnd.integers(0, C, size=len(rest))
    assign[:C] = np.arange(C)          # no empty cluster
    members = [rest[assign == c] for c in range(C)]
    offs = np.zeros(C + 1, dtype=np.uint64)
    offs[1:] = np.cumsum([len(m) for m in members])
    cl_members = np.concatenate(members).astype(np.int64)
    cut = (2 * C) // 3
    groups = [np.arange(cut), np.arange(cut, C)]
    group_offsets, centre_cluster, centres = [0], [], []
    for g in groups:
        for c in rnd.permutation(g):
            centre_cluster.append(int(c))
            centres.append(np.rint(coords[members[c]].mean(0)).astype(np.uint8))
        group_offsets.append(group_offsets[-1] + len(g))
    stash_perm = rnd.permutation(stash)
    return coords, dict(group_offsets=np.array(group_offsets), centre_cluster=np.array(centre_cluster),
                        centres=np.array(centres), cl_offsets=offs, cl_members=cl_members,
                        stash=stash_perm)


def test_clustering_knns_all_clusters_is_brute_force():
    # retrieving every cluster with exact selections (and bins of one centre
    # each, where ApproxTopk degenerates to exact) finds the true k nearest
    from oracle import clustering
    coords, lay = _toy_layout(3000, 12, 30, 1, stash_n=400)
    k = 10
    u = [20, 10]
    for q in inputs.mixture_coords(6, 12, 6, 25.0, 2, means_seed=1):
        bd = clustering.sq_dist(coords, q)
        want = np.sort(bd)[:k]
        for l, l_s in [([0, 0], 0), ([20, 10], 400)]:
            ids = clustering.clustering_knns(q, coords, **lay, k=k, u=u, l=l, l_s=l_s, r_c=0, r_p=0,
                                             maxval=2 ** 31)
            assert np.array_equal(np.sort(bd[ids]), want)
            assert len(set(ids.tolist())) == k


def test_clustering_knns_stash_only_and_truncation():
    # most points in the stash (a linear scan), every cluster retrieved: with
    # r_p > 0 the result holds the k smallest truncated distances
    from oracle import clustering
    coords, lay = _toy_layout(2000, 8, 6, 3, stash_n=1500)
    k = 8
    for r_p in (0, 4):
        for q in inputs.mixture_coords(4, 8, 6, 25.0, 4, means_seed=3):
            ids = clustering.clustering_knns(q, coords, **lay, k=k, u=[4, 2], l=[0, 0], l_s=0, r_c=3,
                                             r_p=r_p, maxval=2 ** 31)
            bd = clustering.sq_dist(coords, q) >> r_p
            assert np.array_equal(np.sort(bd[ids]), np.sort(bd)[:k])


def test_clustering_knns_one_probe_finds_own_cluster_points():
    # u = 1 per group, no stash: the result lies in the union of each group's
    # nearest-centre cluster, and is the exact top-k of that union
    from oracle import clustering
    coords, lay = _toy_layout(1500, 6, 12, 5)
    k = 5
    for q in inputs.mixture_coords(5, 6, 6, 25.0, 6, means_seed=5):
        ids = clustering.clustering_knns(q, coords, **lay, k=k, u=[1, 1], l=[0, 0], l_s=0, r_c=0,
                                         r_p=0, maxval=2 ** 31)
        union = []
        go = lay["group_offsets"]
        for i in range(2):
            cd = clustering.sq_dist(lay["centres"][go[i]:go[i + 1]], q)
            c = lay["centre_cluster"][go[i] + int(np.argmin(cd))]
            union += lay["cl_members"][int(lay["cl_offsets"][c]):int(lay["cl_offsets"][c + 1])].tolist()
        union = np.array(union)
        bd = clustering.sq_dist(coords[union], q)
        assert set(ids.tolist()) <= set(union.tolist())
        assert np.array_equal(np.sort(clustering.sq_dist(coords[ids], q)), np.sort(bd)[:k])


# ---------------------------------------------------------------- slot encoding
@pytest.mark.parametrize("N", [64, 256])
def test_slot_transform_definition_and_ring_isomorphism(N):
    # NTT_t follows the same O(N^2) definition as the RNS transforms, with the
    # smallest primitive 2N-th root mod t; it maps negacyclic products mod t
    # to slot-wise products and constants to constant slots
    O = Oracle(N, 2, 40, 0, 4)
    t = O.t
    assert O.slots_ok and (t - 1) % (2 * N) == 0
    assert pow(O.psi_t, N, t) == t - 1
    rnd = np.random.default_rng(N + 1)
    a = rnd.integers(0, t, size=N, dtype=np.uint64)
    b = rnd.integers(0, t, size=N, dtype=np.uint64)
    fa, fb = O.ntt_t(a), O.ntt_t(b)
    assert [int(v) for v in fa] == _ntt_definition(a, t, O.psi_t)
    assert np.array_equal(O.intt_t(fa), a)
    prod = O.schoolbook_mod(a, b, t)
    assert np.array_equal(O.ntt_t(prod), (fa.astype(object) * fb.astype(object) % t).astype(np.uint64))
    c = np.zeros(N, dtype=np.uint64)
    c[0] = 12345
    assert np.all(O.ntt_t(c) == 12345)


def test_mask_draw_matches_coefficient_shares():
    # the per-position mask value used by the slot shares is the one the
    # coefficient-encoding epilogue draws (share = t - r)
    O = Oracle(256, 2, 40, 0, 5)
    coords = inputs.uniform_coords(600, 5, 3)
    s, s_hat = O.keygen(1)
    ct = O.encrypt(s_hat, inputs.uniform_coords(1, 5, 4)[0], 2, 7)
    _, share = O.distances(ct, coords, None, 9, 7)
    r = np.array([O.mask_r(9, 7, x) for x in range(600)], dtype=np.int64)
    assert np.array_equal(share.astype(np.int64), (O.t - r) % O.t)


@pytest.mark.parametrize("cfg,n", [((256, 2, 40, 0, 5), 700), ((64, 3, 50, 0, 3), 64)])
def test_slot_encoding_shares_reconstruct_brute_force(cfg, n):
    # the whole path in slot encoding: encrypted distances, slot shares on both
    # sides, the sum equals the integer squared distance of every point
    O = Oracle(*cfg)
    d = cfg[4]
    coords = inputs.uniform_coords(n, d, 11)
    perm = inputs.permutation(n, 12)
    qv = inputs.uniform_coords(1, d, 13)[0]
    s, s_hat = O.keygen(5)
    ct = O.encrypt(s_hat, qv, 6, 3)
    out, srv = O.distances(ct, coords, perm, 8, 3, slots=True)
    cli = O.decrypt_shares(out, s, qv, n, slots=True)
    brute = np.sum((coords[perm].astype(np.int64) - qv.astype(np.int64)) ** 2, axis=1)
    assert np.array_equal((cli.astype(np.int64) + srv) % O.t, brute)
    # decrypting slot-encoded responses as coefficients does not give the distances
    cli_coef = O.decrypt_shares(out, s, qv, n)
    assert not np.array_equal((cli_coef.astype(np.int64) + srv) % O.t, brute)


def test_corrupted_response_coefficient_breaks_exactly_its_share():
    # a flipped residue bit of c0 at coefficient x changes the decrypted
    # plaintext at x only: the share reconstruction catches it there
    O = Oracle(256, 2, 40, 0, 5)
    n, x = 600, 137
    coords = inputs.uniform_coords(n, 5, 11)
    qv = inputs.uniform_coords(1, 5, 12)[0]
    s, s_hat = O.keygen(11)
    ct = O.encrypt(s_hat, qv, 13, 11)
    out, srv = O.distances(ct, coords, None, 14, 11)
    brute = np.sum((coords.astype(np.int64) - qv.astype(np.int64)) ** 2, axis=1)
    assert np.array_equal((O.decrypt_shares(out, s, qv, n).astype(np.int64) + srv) % O.t, brute)
    bad = out.copy()
    bad[0, 0, 0, x] ^= np.uint64(1 << 30)
    rec = (O.decrypt_shares(bad, s, qv, n).astype(np.int64) + srv) % O.t
    assert np.flatnonzero(rec != brute).tolist() == [x]


def test_response_equals_textbook_rederivation():
    # The oracle's response blocks re-derived in pure Python from the
    # definition (Sec. 5.3, Pi_ls step 3): c_c = sum_i c_{i,c} * g_i by the
    # schoolbook negacyclic product mod q_j (no NTT), then c_0 += Delta
    # (||p||^2 + r) with Delta = floor(Q / t) and r the mask draw of each
    # position (padding included).  Shares only the coefficient transform
    # (pinned against its O(N^2) definition) and the ChaCha20 draws (RFC 8439).
    N, L, bits, d, n = 64, 2, 40, 3, 100
    O = Oracle(N, L, bits, 0, d)
    qs = [int(x) for x in O.q]
    t = O.t
    Q = 1
    for qj in qs:
        Q *= qj
    Delta = Q // t
    coords = inputs.uniform_coords(n, d, 31)
    perm = inputs.permutation(n, 32)
    qv = inputs.uniform_coords(1, d, 33)[0]
    s, s_hat = O.keygen(34)
    ct = O.encrypt(s_hat, qv, 35, 5)
    out, srv = O.distances(ct, coords, perm, 36, 5)

    def negacyclic(a, b, m):
        res = [0] * N
        for u in range(N):
            if a[u] == 0:
                continue
            for v in range(N):
                w = u + v
                if w < N:
                    res[w] += a[u] * b[v]
                else:
                    res[w - N] -= a[u] * b[v]
        return [x % m for x in res]

    K = -(-n // N)
    for k in range(K):
        pts = [int(perm[k * N + x]) if k * N + x < n else None for x in range(N)]
        for j, qj in enumerate(qs):
            for c in range(2):
                acc = [0] * N
                for i in range(d):
                    a = [int(v) for v in O.intt(ct[i, c, j], j)]
                    g = [int(coords[p][i]) if p is not None else 0 for p in pts]
                    acc = [(x + y) % qj for x, y in zip(acc, negacyclic(a, g, qj))]
                if c == 0:
                    for x in range(N):
                        p = pts[x]
                        nrm = int(np.sum(coords[p].astype(np.int64) ** 2)) if p is not None else 0
                        r = O.mask_r(36, 5, k * N + x)
                        acc[x] = (acc[x] + (Delta % qj) * ((nrm + r) % t)) % qj
                assert [int(v) for v in out[k, c, j]] == acc, (k, j, c)
    # and the server's share is t - r at every database position
    r_all = np.array([O.mask_r(36, 5, x) for x in range(n)], dtype=np.int64)
    assert np.array_equal(srv.astype(np.int64), (t - r_all) % t)


def test_decryption_equals_textbook_rederivation():
    # the client's share re-derived in pure Python: w_j = c0 + c1 s by the
    # schoolbook negacyclic product mod q_j, w by CRT, m = round(t w / Q)
    # mod t, share = m + ||q||^2 mod t
    N, L, bits, d, n = 64, 2, 40, 3, 100
    O = Oracle(N, L, bits, 0, d)
    qs = [int(x) for x in O.q]
    t = O.t
    Q = 1
    for qj in qs:
        Q *= qj
    coords = inputs.uniform_coords(n, d, 41)
    qv = inputs.uniform_coords(1, d, 42)[0]
    s, s_hat = O.keygen(43)
    ct = O.encrypt(s_hat, qv, 44, 6)
    out, _ = O.distances(ct, coords, None, 45, 6)
    got = O.decrypt_shares(out, s, qv, n)
    sv = [int(v) for v in s]
    qn = int(np.sum(qv.astype(np.int64) ** 2))
    want = []
    for k in range(out.shape[0]):
        w_res = []
        for j, qj in enumerate(qs):
            c0 = [int(v) for v in out[k, 0, j]]
            c1 = [int(v) for v in out[k, 1, j]]
            prod = [0] * N
            for u in range(N):
                if sv[u] == 0:
                    continue
                for v in range(N):
                    w = u + v
                    term = sv[u] * c1[v]
                    if w < N:
                        prod[w] += term
                    else:
                        prod[w - N] -= term
            w_res.append([(c0[x] + prod[x]) % qj for x in range(N)])
        for x in range(N):
            w = 0
            for j, qj in enumerate(qs):
                Qj = Q // qj
                w += w_res[j][x] * Qj * pow(Qj, -1, qj)
            w %= Q
            m = ((t * w + Q // 2) // Q) % t
            want.append((m + qn) % t)
    assert got.tolist() == want[:n]


def test_encryption_phase_is_the_documented_error_plus_message():
    # c0 + c1 s (back in coefficient form) is exactly e + Delta m_i: e the
    # centred binomial (eta = 21) of the low 42 bits of draw (seed, 3, qid
    # 2^16 + i) at each coefficient, m_i = (t - 2 q_i) mod t on coefficient 0
    N, L, bits, d = 64, 2, 40, 3
    O = Oracle(N, L, bits, 0, d)
    qs = [int(x) for x in O.q]
    t = O.t
    Q = 1
    for qj in qs:
        Q *= qj
    Delta = Q // t
    qv = inputs.uniform_coords(1, d, 51)[0]
    seed, qid = 52, 7
    s, s_hat = O.keygen(53)
    ct = O.encrypt(s_hat, qv, seed, qid)
    m21 = (1 << 21) - 1
    for i in range(d):
        e = []
        for x in range(N):
            lo, _ = O.draw128(seed, 3, (qid << 16) | i, x)
            e.append(bin(lo & m21).count("1") - bin((lo >> 21) & m21).count("1"))
        m = (t - 2 * int(qv[i])) % t
        for j, qj in enumerate(qs):
            phase = (ct[i, 0, j].astype(object) + ct[i, 1, j].astype(object) * s_hat[j].astype(object)) % qj
            v = [int(a) for a in O.intt(np.array(phase, dtype=np.uint64), j)]
            want = [ex % qj for ex in e]
            want[0] = (want[0] + (Delta % qj) * m) % qj
            assert v == want, (i, j)


@pytest.mark.parametrize("F", [0, 40, 200])
def test_circuit_privacy_terms_equal_textbook_rederivation(F):
    # Sec. 2.3, circuit privacy, re-derived in pure Python at N = 64 with
    # schoolbook products (no NTT): the public key's phase pk0 + pk1 s is its
    # error draw (CBD eta = 21, stream 6); the privacy response minus the plain
    # one is pk_c u in coefficient form, u ternary ((lo mod 3) - 1, stream 7,
    # position k N + x), plus e1 = (low F + 1 bits of the 256-bit value of
    # streams 9 and 10) - 2^F on c0 and e2 = CBD of stream 8 on c1
    N, L, bits, d, n = 64, 2, 40, 2, 100
    O = Oracle(N, L, bits, 0, d)
    qs = [int(x) for x in O.q]
    m21 = (1 << 21) - 1

    def cbd(lo):
        return bin(lo & m21).count("1") - bin((lo >> 21) & m21).count("1")

    def negacyclic(a, b, m):
        res = [0] * N
        for u in range(N):
            for v in range(N):
                w = u + v
                res[w % N] += a[u] * b[v] if w < N else -a[u] * b[v]
        return [x % m for x in res]

    coords = inputs.uniform_coords(n, d, 60)
    qv = inputs.uniform_coords(1, d, 61)[0]
    s, s_hat = O.keygen(62)
    pk = O.public_key(s_hat, 63)
    e_pk = [cbd(O.draw128(63, 6, 0, x)[0]) for x in range(N)]
    for j, qj in enumerate(qs):
        p0 = [int(v) for v in O.intt(pk[0, j], j)]
        p1 = [int(v) for v in O.intt(pk[1, j], j)]
        ph = [(a + b) % qj for a, b in zip(p0, negacyclic(p1, [int(v) % qj for v in s], qj))]
        assert ph == [e % qj for e in e_pk], j
    seed, qid = 64, 9
    ct = O.encrypt(s_hat, qv, 65, qid)
    plain, srv0 = O.distances(ct, coords, None, seed, qid)
    priv, srv = O.distances(ct, coords, None, seed, qid, pk=pk, flood_bits=F)
    assert np.array_equal(srv, srv0)
    for k in range(-(-n // N)):
        pos = [k * N + x for x in range(N)]
        u = [O.draw128(seed, 7, qid, p)[0] % 3 - 1 for p in pos]
        e1, e2 = [], []
        for p in pos:
            a, b = O.draw128(seed, 9, qid, p), O.draw128(seed, 10, qid, p)
            v = a[0] | (a[1] << 64) | (b[0] << 128) | (b[1] << 192)
            e1.append((v & ((1 << (F + 1)) - 1)) - (1 << F))
            e2.append(cbd(O.draw128(seed, 8, qid, p)[0]))
        assert all(-(1 << F) <= e < (1 << F) for e in e1)
        for j, qj in enumerate(qs):
            for c, e in ((0, e1), (1, e2)):
                pkc = [int(v) for v in O.intt(pk[c, j], j)]
                want = [(x + y) % qj for x, y in zip(negacyclic(pkc, [w % qj for w in u], qj), e)]
                diff = [(int(a) - int(b)) % qj for a, b in zip(priv[k, c, j], plain[k, c, j])]
                assert diff == want, (F, k, c, j)


@pytest.mark.parametrize("cfg", [(64, 2, 40, 0, 4), (256, 3, 60, 0, 8)])
def test_maximum_flooding_still_decrypts_worst_case_distances(cfg):
    # Sec. 2.3 noise flooding at the largest exponent allowed, F = floor(log2
    # Delta) - 2 (2^F <= Delta / 4, the rest of the Delta / 2 margin left to
    # the structured noise): extreme coordinates (0 against 255, the largest
    # distance d 255^2 and the largest plaintext overflow) still reconstruct
    # exactly, and the phase noise is the flooding term
    O = Oracle(*cfg)
    N, d = cfg[0], cfg[4]
    n = 2 * N - 3
    coords = np.full((n, d), 255, dtype=np.uint8)
    coords[1::3] = 0
    rnd = np.random.default_rng(cfg[0])
    coords[2::3] = rnd.integers(0, 256, size=coords[2::3].shape, dtype=np.uint8)
    F = O.max_flood_bits()
    assert 2 ** F <= O.P.delta // 4 < 2 ** (F + 1)
    s, s_hat = O.keygen(71)
    pk = O.public_key(s_hat, 72)
    for qv in (np.zeros(d, dtype=np.uint8), np.full(d, 255, dtype=np.uint8)):
        ct = O.encrypt(s_hat, qv, 73, 4)
        out, srv = O.distances(ct, coords, None, 74, 4, pk=pk, flood_bits=F)
        cli = O.decrypt_shares(out, s, qv, n)
        brute = np.sum((coords.astype(np.int64) - qv.astype(np.int64)) ** 2, axis=1)
        assert np.array_equal((cli.astype(np.int64) + srv) % O.t, brute)
        m = O.scale_round(O.decrypt_phase(out, s))
        noise = max(O.phase_noise(out, s, m))
        assert 2 ** (F - 2) <= noise < O.P.delta // 2


def test_encryption_c1_is_the_documented_stream():
    # c1 = a, drawn directly in NTT form: slot s of prime j, coordinate i is
    # (hi 2^64 + lo) mod q_j of draw s of stream (seed, 2, qid 2^16 + j 2^12 + i)
    N, L, bits, d = 64, 2, 40, 3
    O = Oracle(N, L, bits, 0, d)
    s, s_hat = O.keygen(91)
    seed, qid = 92, 6
    ct = O.encrypt(s_hat, inputs.uniform_coords(1, d, 93)[0], seed, qid)
    for i in range(d):
        for j, qj in enumerate(int(x) for x in O.q):
            want = []
            for x in range(N):
                lo, hi = O.draw128(seed, 2, (qid << 16) | (j << 12) | i, x)
                want.append(((hi << 64) | lo) % qj)
            assert [int(v) for v in ct[i, 1, j]] == want, (i, j)


# ------------------------------------------------------- modulus switching

@pytest.mark.parametrize("cfg", [(64, 2, 50, 0, 4), (64, 3, 60, 0, 4), (64, 4, 60, 0, 4)])
def test_mod_switch_removes_errors_below_half_the_dropped_modulus(cfg):
    # round(q_0 c / Q) for c = a (Q / q_0) + e: exactly a whenever |e| is below
    # half of D = Q / q_0 (D is odd, so no ties), including e = 0, both
    # extreme errors and the wrap of negative c below zero
    O = Oracle(*cfg)
    P = O.P
    Q, q0 = P.Q, P.q[0]
    D = Q // q0
    assert D * q0 == Q and D % 2 == 1
    N, L = cfg[0], cfg[1]
    rnd = random.Random(L)
    ct = np.zeros((1, 2, L, N), dtype=np.uint64)
    want = np.zeros((1, 2, N), dtype=np.uint64)
    half = (D - 1) // 2
    for c in range(2):
        for x in range(N):
            a = rnd.randrange(q0) if x > 2 else [0, q0 - 1, 1][x]
            e = [0, half, -half, 1, -1][x % 5] if x < 10 else rnd.randrange(-half, half + 1)
            v = (a * D + e) % Q
            for j, qj in enumerate(P.q):
                ct[0, c, j, x] = v % qj
            want[0, c, x] = a
    assert np.array_equal(O.mod_switch(ct), want)


@pytest.mark.parametrize("cfg,flood,slots", [
    ((64, 2, 40, 0, 4), False, False),
    ((256, 3, 60, 0, 8), False, False),
    ((256, 3, 60, 0, 8), True, False),      # the largest flooding exponent
    ((64, 4, 60, 0, 3), False, False),
    ((256, 2, 40, 0, 5), False, True),      # slot encoding
])
def test_switched_responses_reconstruct_brute_force_distances(cfg, flood, slots):
    # the responses switched down to q_0 and decrypted there: the shares still
    # add up to ||q - p||^2 for every point, with extreme coordinates (the
    # largest distances); the switched response is 1 / L of the bytes
    O = Oracle(*cfg)
    N, L, d = cfg[0], cfg[1], cfg[4]
    n = 2 * N - 3
    coords = np.full((n, d), 255, dtype=np.uint8)
    coords[1::3] = 0
    rnd = np.random.default_rng(N + L)
    coords[2::3] = rnd.integers(0, 256, size=coords[2::3].shape, dtype=np.uint8)
    perm = inputs.permutation(n, 3)
    s, s_hat = O.keygen(31)
    pk = O.public_key(s_hat, 32) if flood else None
    F = O.max_flood_bits() if flood else 0
    for qv in (np.zeros(d, dtype=np.uint8), np.full(d, 255, dtype=np.uint8)):
        ct = O.encrypt(s_hat, qv, 33, 6)
        out, srv = O.distances(ct, coords, perm, 34, 6, pk=pk, flood_bits=F, slots=slots)
        sw = O.mod_switch(out)
        assert sw.nbytes * L == out.nbytes
        cli = O.decrypt_shares_switched(sw, s, qv, n, slots=slots)
        brute = np.sum((coords[perm].astype(np.int64) - qv.astype(np.int64)) ** 2, axis=1)
        assert np.array_equal((cli.astype(np.int64) + srv) % O.t, brute)
