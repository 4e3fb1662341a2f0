"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds none of the method's arithmetic: it only draws databases,
queries, permutations, clusterings and arrival times.  The datasets the paper
evaluates on (SIFT, Deep1B, Amazon; Sec. 7.1 "Datasets") are not available, so
these draws stand in for them with the same n, d and uint8 coordinate range:

* uniform:   coordinates uniform in [0, 255];
* mixture:   a Gaussian mixture with `n_comp` components, means uniform in
             [0, 255]^d, isotropic sigma, optional mixture weights, clipped
             and rounded to uint8;
* clusters:  seeded Lloyd k-means (Sec. 2.5) over mixture data, cluster lists
             as CSR (members ascending), per-query probe lists = the P nearest
             quantised centres (ties to the lower id);
* arrivals:  Poisson arrival times for the serving loop.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence(seed))


def uniform_coords(n: int, d: int, seed: int) -> np.ndarray:
    return rng(seed).integers(0, 256, size=(n, d), dtype=np.uint8)


def mixture_means(d: int, n_comp: int, seed: int) -> np.ndarray:
    return rng(seed).uniform(0.0, 255.0, size=(n_comp, d)).astype(np.float32)


def mixture_coords(n: int, d: int, n_comp: int, sigma: float, seed: int,
                   weights: np.ndarray | None = None, chunk: int = 1 << 18,
                   means_seed: int | None = None) -> np.ndarray:
    """n points of a Gaussian mixture clipped to uint8.  Queries drawn "from the
    same mixture" use the same means_seed with a different seed."""
    means = mixture_means(d, n_comp, seed if means_seed is None else means_seed)
    g = rng(seed + 0x9E3779B9)
    p = None if weights is None else np.asarray(weights, dtype=np.float64) / np.sum(weights)
    out = np.empty((n, d), dtype=np.uint8)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        comp = g.choice(n_comp, size=e - s, p=p)
        x = means[comp] + g.standard_normal(size=(e - s, d)).astype(np.float32) * sigma
        out[s:e] = np.clip(np.rint(x), 0, 255).astype(np.uint8)
    return out


def zipf_weights(n_comp: int, a: float) -> np.ndarray:
    r = np.arange(1, n_comp + 1, dtype=np.float64)
    w = r ** (-a)
    return w / w.sum()


def permutation(n: int, seed: int) -> np.ndarray:
    """The server's random permutation of its points (Alg. 3 first line):
    position x holds original point perm[x]."""
    return rng(seed).permutation(n).astype(np.uint32)


def lloyd_kmeans(x: np.ndarray, k: int, iters: int, seed: int):
    """Plain Lloyd iterations: initial centres = the first k points of a seeded
    permutation; assignment ties go to the lower centre id (argmin)."""
    xf = x.astype(np.float32)
    init = rng(seed).permutation(len(x))[:k]
    c = xf[init].copy()
    xn = np.sum(xf * xf, axis=1)
    assign = np.zeros(len(x), dtype=np.int64)
    for _ in range(iters):
        assign = _assign(xf, xn, c)
        sums = np.zeros_like(c, dtype=np.float64)
        np.add.at(sums, assign, xf)
        cnt = np.bincount(assign, minlength=k)
        nz = cnt > 0
        c[nz] = (sums[nz] / cnt[nz, None]).astype(np.float32)
    assign = _assign(xf, xn, c)
    centres = np.clip(np.rint(c), 0, 255).astype(np.uint8)
    return centres, assign


def _assign(xf, xn, c, chunk: int = 1 << 16):
    cn = np.sum(c * c, axis=1)
    out = np.empty(len(xf), dtype=np.int64)
    for s in range(0, len(xf), chunk):
        e = min(len(xf), s + chunk)
        dist = xn[s:e, None] - 2.0 * (xf[s:e] @ c.T) + cn[None, :]
        out[s:e] = np.argmin(dist, axis=1)
    return out


def clusters_csr(assign: np.ndarray, k: int):
    """CSR lists: members of cluster c are members[offsets[c]:offsets[c+1]],
    ascending point index."""
    order = np.argsort(assign, kind="stable").astype(np.uint32)
    cnt = np.bincount(assign, minlength=k)
    offsets = np.zeros(k + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum(cnt)
    return offsets, order


def probes(queries: np.ndarray, centres: np.ndarray, n_probe: int) -> np.ndarray:
    """Per query, the n_probe nearest quantised centres by exact integer squared
    distance, ties to the lower centre id, nearest first."""
    qi = queries.astype(np.int64)
    ci = centres.astype(np.int64)
    dist = (np.sum(qi * qi, axis=1)[:, None] - 2 * qi @ ci.T
            + np.sum(ci * ci, axis=1)[None, :])
    out = np.empty((len(queries), n_probe), dtype=np.uint32)
    ids = np.arange(len(centres))
    for b in range(len(queries)):
        order = np.lexsort((ids, dist[b]))[:n_probe]
        out[b] = order
    return out


def poisson_arrivals(rate_per_s: float, duration_s: float, seed: int) -> np.ndarray:
    g = rng(seed)
    t, out = 0.0, []
    while True:
        t += g.exponential(1.0 / rate_per_s)
        if t >= duration_s:
            break
        out.append(t)
    return np.array(out, dtype=np.float64)


def mixture_coords_device(n: int, d: int, n_comp: int, sigma: float, seed: int,
                          means_seed: int | None = None, device: str = "cuda",
                          chunk: int = 1 << 22):
    """Large mixture draws on the GPU (seeded torch generator): the same
    distribution as mixture_coords, for databases too big to draw on the host
    in reasonable time.  Returns a uint8 tensor [n][d] on `device`."""
    import torch

    gm = torch.Generator(device="cpu").manual_seed(seed if means_seed is None else means_seed)
    means = (torch.rand((n_comp, d), generator=gm, dtype=torch.float32) * 255.0).to(device)
    g = torch.Generator(device=device).manual_seed(seed + 0x9E3779B9)
    out = torch.empty((n, d), dtype=torch.uint8, device=device)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        comp = torch.randint(0, n_comp, (e - s,), generator=g, device=device)
        x = means[comp] + torch.randn((e - s, d), generator=g, device=device) * sigma
        out[s:e] = x.round_().clamp_(0, 255).to(torch.uint8)
    return out


def permutation_device(n: int, seed: int, device: str = "cuda"):
    import torch

    g = torch.Generator(device=device).manual_seed(seed)
    return torch.randperm(n, generator=g, device=device, dtype=torch.int32).view(torch.uint32)


def mixture_coords_device_weighted(n: int, d: int, n_comp: int, sigma: float, seed: int,
                                   weights, means_seed: int | None = None, device: str = "cuda",
                                   chunk: int = 1 << 22):
    """mixture_coords_device with mixture weights (e.g. Zipf-skewed)."""
    import torch

    gm = torch.Generator(device="cpu").manual_seed(seed if means_seed is None else means_seed)
    means = (torch.rand((n_comp, d), generator=gm, dtype=torch.float32) * 255.0).to(device)
    w = torch.as_tensor(np.asarray(weights, dtype=np.float64), device=device)
    g = torch.Generator(device=device).manual_seed(seed + 0x9E3779B9)
    out = torch.empty((n, d), dtype=torch.uint8, device=device)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        comp = torch.multinomial(w, e - s, replacement=True, generator=g)
        x = means[comp] + torch.randn((e - s, d), generator=g, device=device) * sigma
        out[s:e] = x.round_().clamp_(0, 255).to(torch.uint8)
    return out


def lloyd_kmeans_device(x, k: int, iters: int, seed: int):
    """Lloyd iterations on the GPU in fp32 (data preparation only): initial
    centres = the first k points of a seeded permutation; returns quantised
    centres (uint8 [k][d]) and the final assignment (int64 [n])."""
    import torch

    xf = x.float()
    g = torch.Generator(device=x.device).manual_seed(seed)
    init = torch.randperm(x.shape[0], generator=g, device=x.device)[:k]
    c = xf[init].clone()
    xn = (xf * xf).sum(1)

    def assign(c):
        cn = (c * c).sum(1)
        out = torch.empty(x.shape[0], dtype=torch.int64, device=x.device)
        for s in range(0, x.shape[0], 1 << 18):
            e = min(x.shape[0], s + (1 << 18))
            dist = xn[s:e, None] - 2.0 * (xf[s:e] @ c.T) + cn[None, :]
            out[s:e] = dist.argmin(1)
        return out

    for _ in range(iters):
        a = assign(c)
        sums = torch.zeros_like(c).index_add_(0, a, xf)
        cnt = torch.bincount(a, minlength=k).float()
        nz = cnt > 0
        c[nz] = sums[nz] / cnt[nz, None]
    a = assign(c)
    return c.round().clamp(0, 255).to(torch.uint8), a


def probes_device(queries, centres, n_probe: int):
    """Exact integer squared distances on the GPU; the n_probe nearest centres
    per query, ties to the lower id (stable sort), nearest first."""
    import torch

    # integer inner products below 2^24 are exact in fp64
    qi = queries.double()
    ci = centres.double()
    dist = ((qi * qi).sum(1)[:, None] - 2 * qi @ ci.T + (ci * ci).sum(1)[None, :]).round().long()
    order = torch.sort(dist, dim=1, stable=True).indices[:, :n_probe]
    return order.to(torch.int32)
