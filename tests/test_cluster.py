"""Host logic of the clustering protocol's preprocessing (Sec. 5, balanced
clustering and stash): invariants of the groups, the stash split and the
server's layout, on CPU tensors."""
import numpy as np
import torch

from paper_1904_02033_b300 import cluster, inputs


def _groups(n=6000, d=16, m=120, alpha=0.3, seed=3):
    coords = inputs.mixture_coords(n, d, 8, 22.0, seed)
    return coords, cluster.balanced_clustering(torch.from_numpy(coords), m, alpha, iters=6, seed=seed)


def test_balanced_clustering_partitions_with_bounded_sizes():
    n, m, alpha = 6000, 120, 0.3
    coords, groups = _groups(n=n, m=m, alpha=alpha)
    allm = np.concatenate([mm for g in groups for mm in g.members])
    assert np.array_equal(np.sort(allm), np.arange(n))           # disjoint and covering
    for g in groups:
        assert len(g.members) == g.centres.shape[0]
        assert all(0 < len(mm) <= m for mm in g.members)
        assert all(np.all(np.diff(mm) > 0) for mm in g.members)   # ascending ids
    # each level passes at most an alpha fraction of its points to the next
    left = n
    for g in groups[:-1]:
        nxt = left - sum(len(mm) for mm in g.members)
        assert nxt <= alpha * left + 1e-9
        left = nxt
    assert len(groups) <= 1 + int(np.ceil(np.log(n) / np.log(1 / alpha)))
    # a centre is the rounded mean of its members
    g = groups[0]
    for j in range(0, len(g.members), 7):
        mean = coords[g.members[j]].astype(np.float64).mean(0)
        assert np.max(np.abs(g.centres[j].astype(np.float64) - mean)) <= 0.5 + 1e-3


def test_small_input_is_one_cluster():
    coords = inputs.uniform_coords(50, 4, 1)
    groups = cluster.balanced_clustering(torch.from_numpy(coords), 64, 0.5)
    assert len(groups) == 1 and len(groups[0].members) == 1
    assert np.array_equal(groups[0].members[0], np.arange(50))


def test_stash_split_and_layout():
    coords, groups = _groups()
    sizes = [sum(len(mm) for mm in g.members) for g in groups]
    for s_max in (0, sizes[-1], sum(sizes[1:]), 10 ** 9):
        kept, stash = cluster.split_stash(groups, s_max)
        T = len(kept)
        assert T >= 1 and len(stash) == sum(sizes[T:]) <= max(s_max, 0)
        if T > 1:
            assert len(stash) + sizes[T - 1] > s_max              # no further group fits
        lay = cluster.make_layout(kept, stash, coords.shape[1], seed=9)
        assert lay.group_offsets[-1] == sum(len(g.members) for g in kept) == len(lay.centre_cluster)
        C = len(lay.cl_offsets) - 1
        for i in range(T):
            g0, g1 = lay.group_offsets[i], lay.group_offsets[i + 1]
            ids = lay.centre_cluster[g0:g1]
            base = sum(len(g.members) for g in kept[:i])
            assert np.array_equal(np.sort(ids), np.arange(base, base + g1 - g0))   # a shuffle
            for p in range(g0, g1):
                c = lay.centre_cluster[p]
                assert np.array_equal(lay.centres[p], kept[i].centres[c - base])
                mm = lay.cl_members[int(lay.cl_offsets[c]):int(lay.cl_offsets[c + 1])]
                assert np.array_equal(mm, kept[i].members[c - base])
        assert C == lay.group_offsets[-1]
        assert np.array_equal(np.sort(lay.stash_perm), stash)
        covered = np.concatenate([lay.cl_members, lay.stash_perm])
        assert np.array_equal(np.sort(covered), np.arange(coords.shape[0]))
