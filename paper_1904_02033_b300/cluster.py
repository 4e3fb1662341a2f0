"""Clustering-based k-NNS: the server's preprocessing (balanced clustering
and stash, Sec. 5 "Balanced Clustering and Stash") and the query pipeline of
Algorithm 4 (ClusteringKNNS), every encrypted step and every selection run by
the library's kernels.

Preprocessing (plaintext, on the server's own data, once per dataset):
  * k-means (Lloyd) on the GPU;
  * balanced clustering: for the current point set, the smallest number of
    centres k for which at most an alpha fraction of the points lies in
    clusters larger than m; the clusters of size <= m form one group, the
    points of the larger ones are clustered again, until no cluster exceeds m;
  * the last groups are collapsed into a stash (at most s_max points), searched
    by linear scan.

Query (Algorithm 4 / Pi_cl, with the garbled-circuit selections and the
DORAM retrieval replaced by their plaintext meaning on reconstructed shares):
  1. the client encrypts the query;
  2. encrypted distances to every group's centres (the centres of a group in a
     server-side random order), decrypted by the client; ApproxTopk with u^i
     winners over l^i bins per group on distances >> r_c;
  3. the selected clusters' points, evaluated in one persistent launch
     (gather path); exact top-k on distances >> r_p;
  4. the stash by linear scan (server-side random order); ApproxTopk with k
     winners over l_s bins on distances >> r_p;
  5. the k smallest of the 2k candidates (those of step 3 first).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch

from . import sanns as S


# ---------------------------------------------------------------------------
# preprocessing
# ---------------------------------------------------------------------------
def kmeans(x: torch.Tensor, k: int, iters: int, seed: int):
    """Lloyd iterations on the GPU: initial centres = the first k points of a
    seeded permutation; assignment by smallest squared distance (lower centre
    id on ties).  Returns float centres [k][d] and the assignment [n]."""
    xf = x.float()
    g = torch.Generator(device=x.device).manual_seed(seed)
    c = xf[torch.randperm(x.shape[0], generator=g, device=x.device)[:k]].clone()
    xn = (xf * xf).sum(1)

    def assign(c):
        cn = (c * c).sum(1)
        out = torch.empty(x.shape[0], dtype=torch.int64, device=x.device)
        for s in range(0, x.shape[0], 1 << 17):
            e = min(x.shape[0], s + (1 << 17))
            out[s:e] = (xn[s:e, None] - 2.0 * (xf[s:e] @ c.T) + cn[None, :]).argmin(1)
        return out

    for _ in range(iters):
        a = assign(c)
        sums = torch.zeros_like(c).index_add_(0, a, xf)
        cnt = torch.bincount(a, minlength=k).float()
        nz = cnt > 0
        c[nz] = sums[nz] / cnt[nz, None]
    return c, assign(c)


@dataclasses.dataclass
class Group:
    centres: np.ndarray        # uint8 [k][d], the rounded k-means centres
    members: list              # list of k arrays of point ids (ascending)


def balanced_clustering(x: torch.Tensor, m: int, alpha: float, iters: int = 10, seed: int = 0,
                        max_search: int = 6) -> list:
    """Groups of clusters of size <= m (Sec. 5).  x: uint8 [n][d] on the GPU."""
    assert 0 < alpha < 1 and m >= 1
    groups = []
    ids = torch.arange(x.shape[0], device=x.device)
    level = 0
    while ids.numel():
        n = ids.numel()
        if n <= m:
            c = x[ids].float().mean(0, keepdim=True)
            groups.append(Group(c.round().clamp(0, 255).to(torch.uint8).cpu().numpy(),
                                [np.sort(ids.cpu().numpy())]))
            break

        def trial(k):
            c, a = kmeans(x[ids], k, iters, seed + 1000 * level + k)
            sizes = torch.bincount(a, minlength=k)
            large = sizes > m
            frac = float(sizes[large].sum()) / n
            return frac, c, a, sizes, large

        # smallest k with at most alpha n points in clusters larger than m:
        # doubling from n / m, then bisection (a bounded number of trials)
        lo, hi = 0, max(1, math.ceil(n / m))
        best = trial(hi)
        while best[0] > alpha and hi < n:
            lo, hi = hi, min(n, 2 * hi)
            best = trial(hi)
        for _ in range(max_search):
            if hi - lo <= 1:
                break
            mid = (lo + hi) // 2
            r = trial(mid)
            if r[0] <= alpha:
                hi, best = mid, r
            else:
                lo = mid
        frac, c, a, sizes, large = best
        # a cluster's centre is the mean of its final members
        c = torch.zeros_like(c).index_add_(0, a, x[ids].float()) / sizes.clamp(min=1)[:, None].float()
        small = (~large).nonzero().flatten()
        members, centres = [], []
        a_cpu, ids_cpu = a.cpu().numpy(), ids.cpu().numpy()
        order = np.argsort(a_cpu, kind="stable")
        bounds = np.searchsorted(a_cpu[order], np.arange(sizes.numel() + 1))
        for j in small.cpu().numpy():
            mem = np.sort(ids_cpu[order[bounds[j]:bounds[j + 1]]])
            if len(mem):
                members.append(mem)
                centres.append(c[j])
        groups.append(Group(torch.stack(centres).round().clamp(0, 255).to(torch.uint8).cpu().numpy(),
                            members))
        ids = ids[large[a]]
        level += 1
    return groups


def split_stash(groups: list, s_max: int):
    """Keep the first T groups; the points of the rest form the stash, T the
    smallest index with at most s_max points after it."""
    sizes = [sum(len(mm) for mm in g.members) for g in groups]
    T = len(groups)
    tail = 0
    while T > 1 and tail + sizes[T - 1] <= s_max:
        tail += sizes[T - 1]
        T -= 1
    stash = np.sort(np.concatenate([mm for g in groups[T:] for mm in g.members])) if T < len(groups) \
        else np.zeros(0, dtype=np.int64)
    return groups[:T], stash


# ---------------------------------------------------------------------------
# the server's layout
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Layout:
    """What the server holds after preprocessing (host copies for the
    plaintext reference in the tests)."""
    group_offsets: np.ndarray   # [T + 1] positions of each group in the centre list
    centre_cluster: np.ndarray  # centre position -> global cluster id
    centres: np.ndarray         # uint8 [sum k^i][d], in position order
    cl_offsets: np.ndarray      # [C + 1] CSR over global cluster ids
    cl_members: np.ndarray      # point ids, ascending within a cluster
    stash_perm: np.ndarray      # stash position -> point id


def make_layout(groups: list, stash: np.ndarray, d: int, seed: int) -> Layout:
    rng = np.random.default_rng(np.random.SeedSequence(seed))
    offs, cc, cent, cl_off, cl_mem = [0], [], [], [0], []
    gid0 = 0
    for g in groups:
        k = len(g.members)
        order = rng.permutation(k)           # the server's shuffle of the group's centres
        for j in order:
            cc.append(gid0 + j)
            cent.append(g.centres[j])
        for mm in g.members:
            cl_mem.append(mm.astype(np.uint32))
            cl_off.append(cl_off[-1] + len(mm))
        gid0 += k
        offs.append(offs[-1] + k)
    stash_perm = rng.permutation(stash).astype(np.uint32) if len(stash) else np.zeros(0, np.uint32)
    return Layout(np.array(offs, dtype=np.int64), np.array(cc, dtype=np.int64),
                  np.array(cent, dtype=np.uint8).reshape(-1, d),
                  np.array(cl_off, dtype=np.uint64), np.concatenate(cl_mem), stash_perm)


@dataclasses.dataclass
class Params:
    k: int = 10                 # neighbours returned
    u: tuple = ()               # clusters selected per group
    l: tuple = ()               # bins per group (ApproxTopk over the centres)
    l_s: int = 0                # bins for the stash
    r_c: int = 0                # truncation of centre distances
    r_p: int = 0                # truncation of point distances


class ClusteringServer:
    """The server's encoded state: centre list, clusters (gather path) and
    stash (linear scan), all resident on the GPU."""

    def __init__(self, ctx: S.Context, coords: torch.Tensor, layout: Layout):
        self.ctx, self.layout = ctx, layout
        self.coords = coords
        self.centres_db = S.sanns_encode_db(ctx, torch.from_numpy(layout.centres).cuda())
        self.clusters = S.sanns_clusters_create(ctx, coords, layout.cl_offsets,
                                                torch.from_numpy(layout.cl_members).cuda())
        self.stash_db = (S.sanns_encode_db(ctx, coords, torch.from_numpy(layout.stash_perm).cuda())
                         if len(layout.stash_perm) else None)


def _contig(t: torch.Tensor) -> torch.Tensor:
    return t.contiguous()


def query(server: ClusteringServer, sk: S.SecretKey, q: torch.Tensor, qids: torch.Tensor,
          prm: Params, seeds=(101, 102, 103, 104)) -> np.ndarray:
    """Algorithm 4 for B queries (uint8 [B][d] on the GPU); returns the k
    neighbour ids per query [B][k] (host)."""
    ctx, lay = server.ctx, server.layout
    B = q.shape[0]
    k = prm.k
    ct = S.sanns_encrypt_query(ctx, sk, q, seeds[0], qids)
    # 2. centres: encrypted distances, client shares, ApproxTopk per group
    nc = int(lay.group_offsets[-1])
    out_c, srv_c = S.sanns_distances(ctx, server.centres_db, ct, seeds[1], qids)
    cli_c = S.sanns_decrypt_shares(ctx, sk, out_c, nc, q)
    probes = []
    for i in range(len(lay.group_offsets) - 1):
        g0, g1 = int(lay.group_offsets[i]), int(lay.group_offsets[i + 1])
        u = min(prm.u[i], g1 - g0)
        bins = min(prm.l[i], g1 - g0) if prm.l[i] else 0
        _, pos = S.sanns_topk(ctx, _contig(cli_c[:, g0:g1]), _contig(srv_c[:, g0:g1]), u,
                              max(bins, u) if bins else 0, prm.r_c)
        probes.append(lay.centre_cluster[g0 + pos.cpu().numpy()])
    probes = np.concatenate(probes, axis=1).astype(np.uint32)
    # 3. the selected clusters' points in one persistent launch; exact top-k
    out_g, srv_g, ids_g, n_b, k_b = S.sanns_distances_gather(ctx, server.clusters, ct, probes,
                                                            seeds[2], qids)
    cand_v = np.zeros((B, 2 * k), dtype=np.uint32)
    cand_i = np.zeros((B, 2 * k), dtype=np.int64)
    blk = np.concatenate([[0], np.cumsum(k_b.astype(np.int64))])
    pts = np.concatenate([[0], np.cumsum(n_b.astype(np.int64))])
    maxv = ctx.query()["t"] - 1
    ids_h = ids_g.cpu().numpy() if ids_g is not None else None
    for b in range(B):
        nb = int(n_b[b])
        cand_v[b, :k] = maxv
        cand_i[b, :k] = -1
        if nb:
            cli_g = S.sanns_decrypt_shares(ctx, sk, out_g[blk[b]:blk[b + 1]].unsqueeze(0), nb,
                                           q[b:b + 1])
            kk = min(k, nb)
            dv, dp = S.sanns_topk(ctx, cli_g, _contig(srv_g[pts[b]:pts[b] + nb].unsqueeze(0)), kk,
                                  0, prm.r_p)
            cand_v[b, :kk] = dv[0].cpu().numpy()
            cand_i[b, :kk] = ids_h[pts[b] + dp[0].cpu().numpy()]
    # 4. the stash: linear scan, ApproxTopk
    ns = len(lay.stash_perm)
    if ns:
        out_s, srv_s = S.sanns_distances(ctx, server.stash_db, ct, seeds[3], qids)
        cli_s = S.sanns_decrypt_shares(ctx, sk, out_s, ns, q)
        kk = min(k, ns)
        bins = max(min(prm.l_s, ns), kk) if prm.l_s else 0
        sv, sp = S.sanns_topk(ctx, cli_s, srv_s, kk, bins, prm.r_p)
        cand_v[:, k:k + kk] = sv.cpu().numpy()
        cand_i[:, k:k + kk] = lay.stash_perm[sp.cpu().numpy()]
        cand_v[:, k + kk:] = maxv
        cand_i[:, k + kk:] = -1
    else:
        cand_v[:, k:] = maxv
        cand_i[:, k:] = -1
    # 5. the k smallest of the 2k candidates, those of step 3 first on ties
    zeros = torch.zeros((B, 2 * k), dtype=torch.uint32, device="cuda")
    _, fp = S.sanns_topk(ctx, torch.from_numpy(cand_v).cuda(), zeros, k)
    fp = fp.cpu().numpy()
    return np.take_along_axis(cand_i, fp, axis=1)
