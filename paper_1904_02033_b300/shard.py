"""Sharding the distance step across GPUs, one process per GPU.

The response blocks are independent (block k of the linear-scan protocol,
f_k = sum_i CMult(c_i, p_ik) + r[kN:(k+1)N], depends only on the points of
block k), so a database of K blocks splits into contiguous block ranges, one
per rank.  The only communication is a broadcast of the query ciphertext
from the source rank and a gather of the ranks' response blocks and server
shares back to it; there is no reduction.  Each rank holds only its shard:
its database is encoded from its slice of the permuted point list with the
shard's position base, so the mask is drawn at global positions and the
gathered result is bit-identical to a single-GPU run.
"""
from __future__ import annotations

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


def distances_sharded(compute, ct_in: torch.Tensor, n: int, N: int, L: int, group=None,
                      src: int = 0):
    """Run `compute(ct_in, k0, k1) -> (ct_out [k1-k0][2][L][N] uint64,
    srv_share [p1-p0] uint32)` on every rank for its block range and return
    the concatenated (ct_out [K][2][L][N], srv_share [n]) on `src` (None on the
    other ranks).  ct_in must have the same shape on every rank; its contents
    are taken from `src`."""
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    dist.broadcast(ct_in.view(torch.int64), src, group=group)
    K = -(-n // N)
    k0, k1 = shard_blocks(K, world, rank)
    out, srv = compute(ct_in, k0, k1)
    # pad to the largest shard so that every rank sends equal-sized tensors
    kmax = max(shard_blocks(K, world, r)[1] - shard_blocks(K, world, r)[0] for r in range(world))
    pbuf = torch.zeros((kmax, 2, L, N), dtype=torch.int64, device=ct_in.device)
    sbuf = torch.zeros(kmax * N, dtype=torch.int32, device=ct_in.device)
    if k1 > k0:
        pbuf[: k1 - k0] = out.reshape(k1 - k0, 2, L, N).view(torch.int64)
        sbuf[: srv.numel()] = srv.view(torch.int32)
    glist = [torch.empty_like(pbuf) for _ in range(world)] if rank == src else None
    slist = [torch.empty_like(sbuf) for _ in range(world)] if rank == src else None
    dist.gather(pbuf, glist, dst=src, group=group)
    dist.gather(sbuf, slist, dst=src, group=group)
    if rank != src:
        return None
    outs, srvs = [], []
    for r in range(world):
        a, b = shard_blocks(K, world, r)
        p0, p1 = shard_positions(n, N, a, b)
        outs.append(glist[r][: b - a])
        srvs.append(slist[r][: p1 - p0])
    return (torch.cat(outs).view(torch.uint64).view(K, 2, L, N),
            torch.cat(srvs).view(torch.uint32))


def gpu_shard_compute(ctx, coords: torch.Tensor, perm: torch.Tensor, n: int, mask_seed: int,
                      qids: torch.Tensor):
    """The per-rank compute step on the GPU: encode the rank's slice of the
    permuted list as its own database (position base k0 N) and run the
    distance step on it."""
    from . import sanns as S

    def compute(ct_in, k0, k1):
        p0, p1 = shard_positions(n, ctx.N, k0, k1)
        if p1 <= p0:
            return (torch.empty((0, 2, ctx.L, ctx.N), dtype=torch.uint64, device=ct_in.device),
                    torch.empty(0, dtype=torch.uint32, device=ct_in.device))
        db = S.sanns_encode_db(ctx, coords, perm[p0:p1].contiguous())
        S.sanns_db_set_position_base(db, k0 * ctx.N)
        out, srv = S.sanns_distances(ctx, db, ct_in, mask_seed, qids)
        return out[0], srv[0]

    return compute
