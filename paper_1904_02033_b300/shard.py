"""Sharding the distance step across GPUs, one process per GPU.

The response blocks are independent (block k of the linear-scan protocol,
f_k = sum_i CMult(c_i, p_ik) + r[kN:(k+1)N], depends only on the points of
block k), so a database of K blocks splits into contiguous block ranges, one
per rank.  The only communication is a broadcast of the query ciphertexts
from the source rank and a gather of the ranks' response blocks and server
shares back to it; there is no reduction.  Each rank holds only its shard:
its database is encoded from its slice of the permuted point list with the
shard's position base, so the mask is drawn at global positions and the
gathered result is bit-identical to a single-GPU run.  This holds for any
number of queries per call and for both the per-query and the tensor-core
(batched) distance paths.

The clustering protocol's gather (Algorithm 4: each query's retrieved
clusters scanned as one list) shards its work list by query: every query's
list is evaluated whole on one rank (its mask is drawn at its own list
positions, so it does not depend on which other queries share the call),
and the queries are spread over the ranks by their number of work items
(longest first onto the least-loaded rank).
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def shard_blocks(K: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous, balanced block range [k0, k1) of `rank` among `world`."""
    base, extra = divmod(K, world)
    k0 = rank * base + min(rank, extra)
    return k0, k0 + base + (1 if rank < extra else 0)


def shard_positions(n: int, N: int, k0: int, k1: int) -> tuple[int, int]:
    """Positions [p0, p1) of the points held by blocks [k0, k1)."""
    return min(n, k0 * N), min(n, k1 * N)


def assign_queries(items, world: int) -> list[list[int]]:
    """Queries to ranks by work: longest first onto the least-loaded rank
    (ties to the lower rank); each rank's queries in ascending order."""
    items = np.asarray(items, dtype=np.int64)
    order = sorted(range(len(items)), key=lambda b: (-int(items[b]), b))
    load = [0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for b in order:
        r = min(range(world), key=lambda x: (load[x], x))
        out[r].append(b)
        load[r] += int(items[b])
    return [sorted(q) for q in out]


def _as_signed(t: torch.Tensor) -> torch.Tensor:
    """Same bits as a signed type the collectives move (uint64 -> int64,
    uint32 -> int32)."""
    if t.dtype == torch.uint64:
        return t.view(torch.int64)
    if t.dtype == torch.uint32:
        return t.view(torch.int32)
    return t


def _gather_rows(t: torch.Tensor, rows_per_rank: list[int], group, src: int):
    """Gather a tensor whose leading dimension differs per rank (given on every
    rank by rows_per_rank) to `src`: padded to the largest, trimmed there."""
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    rmax = max(rows_per_rank) if rows_per_rank else 0
    shape = (rmax,) + tuple(t.shape[1:])
    buf = torch.zeros(shape, dtype=_as_signed(t).dtype, device=t.device)
    if t.shape[0]:
        buf[: t.shape[0]] = _as_signed(t)
    glist = [torch.empty_like(buf) for _ in range(world)] if rank == src else None
    dist.gather(buf, glist, dst=src, group=group)
    if rank != src:
        return None
    return [g[:r].view(t.dtype) for g, r in zip(glist, rows_per_rank)]


def distances_sharded(compute, ct_in: torch.Tensor, n: int, N: int, L: int, group=None,
                      src: int = 0):
    """Run `compute(ct_in, k0, k1) -> (ct_out [B][k1-k0][2][L][N] uint64,
    srv_share [B][p1-p0] uint32)` on every rank for its block range and
    return the concatenated (ct_out [B][K][2][L][N], srv_share [B][n]) on
    `src` (None on the other ranks).  ct_in [B][d][2][L][N] must have the
    same shape on every rank; its contents are taken from `src`."""
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    dist.broadcast(_as_signed(ct_in), src, group=group)
    B = ct_in.shape[0]
    K = -(-n // N)
    ranges = [shard_blocks(K, world, r) for r in range(world)]
    k0, k1 = ranges[rank]
    out, srv = compute(ct_in, k0, k1)
    out = _as_signed(out).reshape(B, k1 - k0, 2, L, N)
    srv = _as_signed(srv).reshape(B, -1)
    # block-major for the gather: [k1-k0][B][2][L][N] and [p1-p0][B]
    outs = _gather_rows(out.transpose(0, 1).contiguous(), [b - a for a, b in ranges], group, src)
    pos = [shard_positions(n, N, a, b) for a, b in ranges]
    srvs = _gather_rows(srv.transpose(0, 1).contiguous(), [p1 - p0 for p0, p1 in pos], group, src)
    if rank != src:
        return None
    return (torch.cat(outs).transpose(0, 1).contiguous().view(torch.uint64),
            torch.cat(srvs).transpose(0, 1).contiguous().view(torch.uint32))


def gather_sharded(compute, ct_in: torch.Tensor, blocks_b, points_b, group=None, src: int = 0):
    """The clustering gather sharded by query.  `compute(ct_sub, qs) ->
    (ct_out [sum K_b][2][L][N], srv_share [sum n_b], ids [sum n_b] or None)`
    evaluates the ascending query subset qs (ct_sub = ct_in[qs]) as one
    gather call; blocks_b and points_b (host) are every query's list blocks
    K_b and points n_b.  Returns the single-call layout (all queries in
    order) on `src`, None elsewhere."""
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    dist.broadcast(_as_signed(ct_in), src, group=group)
    blocks_b = np.asarray(blocks_b, dtype=np.int64)
    points_b = np.asarray(points_b, dtype=np.int64)
    assign = assign_queries(blocks_b, world)
    qs = assign[rank]
    if qs:
        idx = torch.as_tensor(qs, dtype=torch.int64, device=ct_in.device)
        out, srv, ids = compute(_as_signed(ct_in)[idx].contiguous().view(torch.uint64), qs)
    else:
        out = torch.empty((0,) + tuple(ct_in.shape[2:]), dtype=torch.uint64, device=ct_in.device)
        srv = torch.empty(0, dtype=torch.uint32, device=ct_in.device)
        ids = None
    with_ids = ids is not None
    if not with_ids:
        ids = torch.zeros_like(srv)
    kb = [int(blocks_b[a].sum()) for a in assign]
    nb = [int(points_b[a].sum()) for a in assign]
    outs = _gather_rows(out, kb, group, src)
    srvs = _gather_rows(srv, nb, group, src)
    idss = _gather_rows(ids, nb, group, src)
    if rank != src:
        return None
    # each rank's concatenation split per query, then all queries in order
    piece_out, piece_srv, piece_ids = {}, {}, {}
    for r, a in enumerate(assign):
        ko = no = 0
        for b in a:
            piece_out[b] = outs[r][ko:ko + blocks_b[b]]
            piece_srv[b] = srvs[r][no:no + points_b[b]]
            piece_ids[b] = idss[r][no:no + points_b[b]]
            ko += int(blocks_b[b])
            no += int(points_b[b])
    B = len(blocks_b)

    def cat(pieces, dtype):
        return torch.cat([_as_signed(p) for p in pieces]).view(dtype)

    cat_out = cat([piece_out[b] for b in range(B)], torch.uint64) if B else out
    cat_srv = cat([piece_srv[b] for b in range(B)], torch.uint32) if B else srv
    cat_ids = cat([piece_ids[b] for b in range(B)], torch.uint32) if B and with_ids else None
    return cat_out, cat_srv, cat_ids


class ShardDatabase:
    """This rank's block range [k0, k1) of a database on its GPU, encoded once
    from its slice of the permuted point list with the position base k0 N
    (and prepared for the tensor-core path when `batched`)."""

    def __init__(self, ctx, coords: torch.Tensor, perm: torch.Tensor, n: int, k0: int, k1: int,
                 batched: bool = False):
        from . import sanns as S

        self.ctx, self.n, self.k0, self.k1, self.batched = ctx, n, k0, k1, batched
        self.p0, self.p1 = shard_positions(n, ctx.N, k0, k1)
        self.db = None
        if self.p1 > self.p0:
            self.db = S.sanns_encode_db(ctx, coords, perm[self.p0:self.p1].contiguous())
            S.sanns_db_set_position_base(self.db, k0 * ctx.N)
            if batched:
                S.sanns_db_prepare_batched(ctx, self.db)

    def distances(self, ct_in: torch.Tensor, mask_seed: int, qids: torch.Tensor, stream=None):
        """(ct_out [B][k1-k0][2][L][N], srv_share [B][p1-p0]) of this shard."""
        from . import sanns as S

        B, ctx = ct_in.shape[0], self.ctx
        if self.db is None:
            return (torch.empty((B, 0, 2, ctx.L, ctx.N), dtype=torch.uint64, device=ct_in.device),
                    torch.empty((B, 0), dtype=torch.uint32, device=ct_in.device))
        if self.batched:
            return S.sanns_distances_batched(ctx, self.db, ct_in, mask_seed, qids, stream=stream)
        return S.sanns_distances(ctx, self.db, ct_in, mask_seed, qids, stream=stream)


def gpu_shard_compute(ctx, coords: torch.Tensor, perm: torch.Tensor, n: int, mask_seed: int,
                      qids: torch.Tensor, batched: bool = False):
    """The per-rank compute step on the GPU for distances_sharded: the rank's
    shard database (encoded on first use, then kept) and the distance step
    on it for all B queries, on the per-query or the tensor-core path."""
    shards: dict = {}

    def compute(ct_in, k0, k1):
        if (k0, k1) not in shards:
            shards[(k0, k1)] = ShardDatabase(ctx, coords, perm, n, k0, k1, batched)
        return shards[(k0, k1)].distances(ct_in, mask_seed, qids)

    return compute


def gpu_gather_compute(ctx, cl, probes, mask_seed: int, qids: torch.Tensor):
    """The per-rank compute step on the GPU for gather_sharded: one
    sanns_distances_gather call over the rank's queries (their probe rows and
    query ids)."""
    from . import sanns as S

    probes = np.ascontiguousarray(probes, dtype=np.uint32)

    def compute(ct_sub, qs):
        idx = torch.as_tensor(qs, dtype=torch.int64, device=qids.device)
        sub_qids = qids.view(torch.int64)[idx].contiguous().view(torch.uint64)
        out, srv, ids, _, _ = S.sanns_distances_gather(ctx, cl, ct_sub, probes[qs], mask_seed, sub_qids)
        return out, srv, ids

    return compute
