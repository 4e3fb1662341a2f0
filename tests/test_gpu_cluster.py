"""The clustering protocol end to end (Algorithm 4 through the library's calls:
encrypted centre distances, per-group ApproxTopk, one gather launch over the
selected clusters, exact top-k, the stash by linear scan, the final top-k),
against the oracle's plaintext Algorithm 4 on the same layout, id for id, and
its 10-NN accuracy against brute force."""
import numpy as np
import pytest
import torch

from oracle import clustering
from paper_1904_02033_b300 import cluster, inputs
from paper_1904_02033_b300 import sanns as S

pytestmark = pytest.mark.gpu


def _setup(cfg, n, d, s_max, seed=5, batched_min=16, batched_min_blocks=128):
    coords = inputs.mixture_coords(n, d, 16, 20.0, seed)
    # the layout is the server's preprocessing, built here on CPU tensors
    groups = cluster.balanced_clustering(torch.from_numpy(coords), 300, 0.3, iters=8, seed=1)
    kept, stash = cluster.split_stash(groups, s_max)
    lay = cluster.make_layout(kept, stash, d, seed=7)
    ctx = S.sanns_ctx_create(*cfg)
    srv = cluster.ClusteringServer(ctx, torch.from_numpy(coords).cuda(), lay, batched_min=batched_min,
                                   batched_min_blocks=batched_min_blocks)
    return coords, lay, ctx, srv


def _oracle_ids(coords, lay, q, prm, t):
    return clustering.clustering_knns(q, coords, lay.group_offsets, lay.centre_cluster, lay.centres,
                                      lay.cl_offsets, lay.cl_members.astype(np.int64),
                                      lay.stash_perm.astype(np.int64), prm.k, prm.u, prm.l, prm.l_s,
                                      prm.r_c, prm.r_p, t - 1)


@pytest.mark.parametrize("cfg,s_max,batched_min", [((4096, 2, 54, 0, 32), 2000, 16),
                                                   ((8192, 3, 60, 0, 32), 0, 16),
                                                   ((8192, 3, 60, 0, 32), 3000, 1)])   # tensor-core path
def test_clustering_query_matches_oracle(cfg, s_max, batched_min):
    n, d, B = 20000, 32, 6
    coords, lay, ctx, srv = _setup(cfg, n, d, s_max, batched_min=batched_min, batched_min_blocks=1)
    T = len(lay.group_offsets) - 1
    sizes = np.diff(lay.group_offsets)
    t = ctx.query()["t"]
    sk = S.sanns_keygen(ctx, 11)
    q = inputs.mixture_coords(B, d, 16, 20.0, 6, means_seed=5)
    qids = torch.from_numpy(np.arange(B, dtype=np.uint64)).cuda()

    def pad(v, fill):
        return tuple((list(v) + [fill] * T)[:T])

    prms = [
        cluster.Params(k=10, u=pad([8, 4], 2), l=pad([24, 12], 4), l_s=300, r_c=0, r_p=0),
        cluster.Params(k=10, u=pad([8, 4], 2), l=pad([0, 0], 0), l_s=0, r_c=2, r_p=3),
        cluster.Params(k=10, u=pad([8, 4], 3), l=pad([0, 12], 0), l_s=50, r_c=1, r_p=2),
        # more than 32 winners per group: the shared-memory sort selection
        cluster.Params(k=40, u=pad([min(40, sizes[0]), 4], 2), l=pad([min(60, sizes[0]), 0], 0),
                       l_s=100, r_c=1, r_p=0),
    ]
    for prm in prms:
        got = cluster.query(srv, sk, torch.from_numpy(q).cuda(), qids, prm)
        for b in range(B):
            want = _oracle_ids(coords, lay, q[b], prm, t)
            assert np.array_equal(got[b], want), (prm, b)


def test_clustering_accuracy_against_brute_force():
    n, d, B, k = 20000, 32, 16, 10
    cfg = (4096, 2, 54, 0, 32)
    coords, lay, ctx, srv = _setup(cfg, n, d, 2000)
    T = len(lay.group_offsets) - 1
    sk = S.sanns_keygen(ctx, 12)
    q = inputs.mixture_coords(B, d, 16, 20.0, 8, means_seed=5)
    qids = torch.from_numpy(np.arange(100, 100 + B, dtype=np.uint64)).cuda()
    u = tuple(([8, 4] + [2] * T)[:T])
    l = tuple(([24, 12] + [4] * T)[:T])
    got = cluster.query(srv, sk, torch.from_numpy(q).cuda(), qids, cluster.Params(k, u, l, 300, 0, 0))
    acc = 0.0
    for b in range(B):
        bd = clustering.sq_dist(coords, q[b])
        kth = np.sort(bd)[k - 1]
        assert np.all(got[b] >= 0) and len(set(got[b].tolist())) == k
        acc += np.sum(bd[got[b]] <= kth) / k
    assert acc / B >= 0.9, acc / B


@pytest.mark.parametrize("F,slots", [(100, False), (0, True), (148, True)])
def test_clustering_query_with_privacy_and_slots(F, slots):
    # circuit privacy and slot encoding change the ciphertexts, not the
    # reconstructed distances: the returned ids are the oracle's
    n, d, B = 20000, 32, 4
    cfg = (8192, 3, 60, 0, 32)
    coords = inputs.mixture_coords(n, d, 16, 20.0, 5)
    groups = cluster.balanced_clustering(torch.from_numpy(coords), 300, 0.3, iters=8, seed=1)
    kept, stash = cluster.split_stash(groups, 2000)
    lay = cluster.make_layout(kept, stash, d, seed=7)
    ctx = S.sanns_ctx_create(*cfg)
    S.sanns_set_encoding(ctx, slots)
    sk = S.sanns_keygen(ctx, 13)
    if F:
        S.sanns_set_circuit_privacy(ctx, S.sanns_public_key(ctx, sk, 14), F)
    srv = cluster.ClusteringServer(ctx, torch.from_numpy(coords).cuda(), lay)
    T = len(lay.group_offsets) - 1
    prm = cluster.Params(k=10, u=tuple(([8, 4] + [2] * T)[:T]), l=tuple(([24, 12] + [4] * T)[:T]),
                         l_s=300, r_c=1, r_p=2)
    q = inputs.mixture_coords(B, d, 16, 20.0, 9, means_seed=5)
    qids = torch.from_numpy(np.arange(B, dtype=np.uint64) + 50).cuda()
    got = cluster.query(srv, sk, torch.from_numpy(q).cuda(), qids, prm)
    t = ctx.query()["t"]
    for b in range(B):
        assert np.array_equal(got[b], _oracle_ids(coords, lay, q[b], prm, t)), b
