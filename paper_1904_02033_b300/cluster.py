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
import time

import numpy as np
import torch

from . import sanns as S


# ---------------------------------------------------------------------------
# preprocessing
# ---------------------------------------------------------------------------
def kmeans(x: torch.Tensor, k: int, iters: int, seed: int):
    """Lloyd iterations (on the GPU in TF32): initial centres = the first k points of a
    seeded permutation; assignment by smallest squared distance (lower centre
    id on ties).  Returns float centres [k][d] and the assignment [n]."""
    if x.is_cuda and not torch.backends.cuda.matmul.allow_tf32:
        # the assignment products on the tensor cores in TF32 (uint8 inputs
        # are exact; the centres round to 10 mantissa bits)
        torch.backends.cuda.matmul.allow_tf32 = True
        try:
            return kmeans(x, k, iters, seed)
        finally:
            torch.backends.cuda.matmul.allow_tf32 = False
    xf = x.float()
    g = torch.Generator(device=x.device).manual_seed(seed)
    c = xf[torch.randperm(x.shape[0], generator=g, device=x.device)[:k]].clone()
    xn = (xf * xf).sum(1)

    def assign(c):
        cn = (c * c).sum(1)
        out = torch.empty(x.shape[0], dtype=torch.int64, device=x.device)
        rows = max(1024, (1 << 27) // c.shape[0])     # a distance tile of at most 512 MB
        for s in range(0, x.shape[0], rows):
            e = min(x.shape[0], s + rows)
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

    def __init__(self, ctx: S.Context, coords: torch.Tensor, layout: Layout, batched_min: int = 16,
                 batched_min_blocks: int = 128):
        """From batched_min queries per call on, the centre and stash
        distances of a list of at least batched_min_blocks blocks run on the
        tensor-core batched path (bit-identical results; needs d <= 128).  Its
        per-call expansion of the queries (proportional to B d N L) pays back
        only over many blocks, so short lists stay on the per-query path."""
        self.ctx, self.layout = ctx, layout
        self.coords = coords
        self.centres_db = S.sanns_encode_db(ctx, torch.from_numpy(layout.centres).cuda())
        self.clusters = S.sanns_clusters_create(ctx, coords, layout.cl_offsets,
                                                torch.from_numpy(layout.cl_members).cuda())
        self.stash_db = (S.sanns_encode_db(ctx, coords, torch.from_numpy(layout.stash_perm).cuda())
                         if len(layout.stash_perm) else None)
        self.batched_min = batched_min if ctx.d <= 128 else 0
        self.batched_dbs = set()
        if self.batched_min:
            for db in (self.centres_db, self.stash_db):
                if db is not None and db.K >= batched_min_blocks:
                    S.sanns_db_prepare_batched(ctx, db)
                    self.batched_dbs.add(id(db))

    def distances(self, db, ct, seed, qids, stream=None):
        B = ct.shape[0]
        if id(db) in self.batched_dbs and B >= self.batched_min:
            return S.sanns_distances_batched(self.ctx, db, ct, seed, qids, stream=stream)
        return S.sanns_distances(self.ctx, db, ct, seed, qids, stream=stream)


class _Stages:
    """Optional per-stage wall clock (device synchronised at each mark)."""

    def __init__(self, out):
        self.out = out
        self.t = time.perf_counter() if out is not None else 0.0

    def mark(self, name):
        if self.out is None:
            return
        torch.cuda.synchronize()
        now = time.perf_counter()
        self.out[name] = self.out.get(name, 0.0) + (now - self.t) * 1e3
        self.t = now


def query(server: ClusteringServer, sk: S.SecretKey, q: torch.Tensor, qids: torch.Tensor,
          prm: Params, seeds=(101, 102, 103, 104), stream=None, timings: dict | None = None) -> np.ndarray:
    """Algorithm 4 for B queries (uint8 [B][d] on the GPU); returns the k
    neighbour ids per query [B][k] (host; -1 where fewer than k points were
    searched).  A dict passed as `timings` accumulates milliseconds per stage
    (the device is synchronised between stages)."""
    st_ = _Stages(timings)
    ctx, lay = server.ctx, server.layout
    B, k, N = q.shape[0], prm.k, ctx.N
    ar = np.arange(B, dtype=np.uint64)
    ct = S.sanns_encrypt_query(ctx, sk, q, seeds[0], qids, stream=stream)
    st_.mark("encrypt")
    # 2. centres: encrypted distances, client shares, ApproxTopk per group
    nc = int(lay.group_offsets[-1])
    out_c, srv_c = server.distances(server.centres_db, ct, seeds[1], qids, stream=stream)
    st_.mark("centres_distances")
    cli_c = S.sanns_decrypt_shares(ctx, sk, out_c, nc, q, stream=stream)
    st_.mark("centres_decrypt")
    # every (group, query) list in one call per selection mode (ApproxTopk
    # where the group has bins, exact where it has none)
    T = len(lay.group_offsets) - 1
    g0s, g1s = lay.group_offsets[:-1].astype(np.int64), lay.group_offsets[1:].astype(np.int64)
    us = np.minimum(np.asarray(prm.u[:T], dtype=np.int64), g1s - g0s)
    ls = np.array([max(min(int(prm.l[i]), int(g1s[i] - g0s[i])), int(us[i])) if prm.l[i] else 0
                   for i in range(T)], dtype=np.int64)
    cols = [None] * T
    for approx in (True, False):
        grp = [i for i in range(T) if (ls[i] > 0) == approx]
        if not grp:
            continue
        gi = np.repeat(np.array(grp), B)                      # segment = (group, query)
        bi = np.tile(np.arange(B, dtype=np.int64), len(grp))
        off = bi * nc + g0s[gi]
        kmax = int(us[grp].max())
        _, pos = S.sanns_topk_segments(ctx, cli_c, srv_c, off, off, (g1s - g0s)[gi], kmax,
                                       int(ls[grp].max()) if approx else 0, prm.r_c,
                                       k_seg=us[gi], bins_seg=ls[gi] if approx else None,
                                       stream=stream)
        pos = pos.cpu().numpy().reshape(len(grp), B, kmax)
        for r, i in enumerate(grp):
            cols[i] = lay.centre_cluster[g0s[i] + pos[r, :, :us[i]]]
    probes = np.concatenate(cols, axis=1).astype(np.uint32)
    st_.mark("centres_select")
    # 3. the selected clusters' points in one persistent launch; every
    #    response block decrypted in one call (block j of query b carries
    #    query b's norm); exact top-k over the B ragged lists
    out_g, srv_g, ids_g, n_b, k_b = S.sanns_distances_gather(ctx, server.clusters, ct, probes,
                                                            seeds[2], qids, stream=stream)
    st_.mark("gather")
    kb = k_b.astype(np.int64)
    blk = np.concatenate([[0], np.cumsum(kb)])
    pts = np.concatenate([[0], np.cumsum(n_b.astype(np.int64))])
    if blk[-1]:
        owner = torch.from_numpy(np.repeat(np.arange(B), kb)).to(q.device)
        cli_g = S.sanns_decrypt_shares(ctx, sk, out_g.unsqueeze(1), N, q.index_select(0, owner),
                                       stream=stream)
    else:   # nothing gathered (only empty clusters selected)
        cli_g = srv_g = torch.zeros(1, dtype=torch.uint32, device=q.device)
    st_.mark("gather_decrypt")
    dv_c, dp_c = S.sanns_topk_segments(ctx, cli_g, srv_g, blk[:-1] * N, pts[:-1], n_b, k, 0, prm.r_p,
                                       stream=stream)
    st_.mark("gather_select")
    # 4. the stash: linear scan, ApproxTopk (fills past the stash's size)
    ns = len(lay.stash_perm)
    if ns:
        out_s, srv_s = server.distances(server.stash_db, ct, seeds[3], qids, stream=stream)
        cli_s = S.sanns_decrypt_shares(ctx, sk, out_s, ns, q, stream=stream)
        bins = max(min(prm.l_s, ns), min(k, ns)) if prm.l_s else 0
        bins = bins if bins >= k else 0     # fewer than k bins: every stash point is a candidate
        off = ar * ns
        dv_s, dp_s = S.sanns_topk_segments(ctx, cli_s, srv_s, off, off, np.full(B, ns), k, bins,
                                           prm.r_p, stream=stream)
    else:
        z = torch.zeros(1, dtype=torch.uint32, device=q.device)
        dv_s, dp_s = S.sanns_topk_segments(ctx, z, z, np.zeros(B), np.zeros(B), np.zeros(B), k,
                                           stream=stream)
    st_.mark("stash")
    # 5. the k smallest of the 2k candidates (cluster candidates first on
    #    ties), as shares (candidate value, 0).  A fill value 2^32 - 1
    #    reconstructs to 2^32 - 1 - t, above every distance (t < 2^31).
    cand = torch.cat([dv_c, dv_s], dim=1).contiguous()
    zeros = torch.zeros_like(cand)
    _, fp = S.sanns_topk(ctx, cand, zeros, k, stream=stream)
    fp = fp.cpu().numpy()
    pc, ps = dp_c.cpu().numpy(), dp_s.cpu().numpy()
    ids_h = ids_g.cpu().numpy().astype(np.int64) if ids_g is not None else None
    out = np.full((B, k), -1, dtype=np.int64)
    for b in range(B):
        for r in range(k):
            j = int(fp[b, r])
            p = int(pc[b, j]) if j < k else int(ps[b, j - k])
            if p < 0:
                continue
            out[b, r] = ids_h[pts[b] + p] if j < k else int(lay.stash_perm[p])
    st_.mark("final")
    return out
