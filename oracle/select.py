"""Plaintext meaning of the selection steps (the paper runs them inside
garbled circuits, which are out of scope here).

TEST INFRASTRUCTURE ONLY (the oracle).

* naive_topk      -- Algorithm 1 (NaiveTopk): k slots, each input inserted by
                     a chain of compare-and-swap steps with strict '<'.
* approx_topk     -- Algorithm 2 (ApproxTopk): l bins of consecutive
                     (already shuffled) positions, the minimum of each bin,
                     then NaiveTopk over the l minima.
* exact_topk      -- the k smallest (value, position) pairs: the same values
                     as naive_topk (its compare-and-swap chain re-inserts a
                     displaced element after equal ones, so its order among
                     equal values is not positional); used where the O(nk)
                     loop is too slow and as the deterministic definition.
* approx_topk_by_position -- Algorithm 2 with that definition for the final
                     selection: bin minima (earlier position on ties), then
                     the k smallest (value, position) of the minima.
* expected_hits   -- E|I| for ApproxTopk under the random-order assumption of
                     Theorem 1, for fixed bin sizes (hypergeometric form).
"""
from __future__ import annotations

import math

import numpy as np


def naive_topk(values, ids, k: int):
    """Algorithm 1 written out: OPT starts as [MAXVAL]*k; every (x, id) walks
    the k slots and swaps in wherever x < OPT[j]."""
    maxval = float("inf")
    opt = [maxval] * k
    idl = [0] * k
    for x, idx in zip(values, ids):
        x = int(x)
        idx = int(idx)
        for j in range(k):
            if x < opt[j]:
                opt[j], x = x, opt[j]
                idl[j], idx = idx, idl[j]
    return opt, idl


def exact_topk(values: np.ndarray, ids: np.ndarray, k: int):
    """The k smallest (value, position) pairs, ascending.  Algorithm 1 selects
    the same values; among equal values its order (and, at the k-th value,
    its choice) can differ."""
    values = np.asarray(values, dtype=np.int64)
    order = np.lexsort((np.arange(len(values)), values))[:k]
    return values[order].tolist(), np.asarray(ids)[order].tolist()


def bin_of(n: int, l: int) -> np.ndarray:
    """Bin index of each position: position x goes to bin floor(x l / n), so the
    l bins are runs of consecutive positions of size floor(n/l) or ceil(n/l)."""
    x = np.arange(n, dtype=np.int64)
    return (x * l) // n


def approx_topk(values: np.ndarray, ids: np.ndarray, k: int, l: int):
    """Algorithm 2: per-bin minimum (ties to the earlier position), then
    NaiveTopk of the l minima."""
    values = np.asarray(values, dtype=np.int64)
    ids = np.asarray(ids)
    n = len(values)
    b = bin_of(n, l)
    mins, mids = [], []
    start = 0
    for i in range(l):
        end = start
        while end < n and b[end] == i:
            end += 1
        seg = values[start:end]
        r = int(np.argmin(seg))  # first minimum
        mins.append(int(seg[r]))
        mids.append(int(ids[start + r]))
        start = end
    return naive_topk(mins, mids, k)


def approx_topk_by_position(values: np.ndarray, ids: np.ndarray, k: int, l: int):
    """Algorithm 2's bins and per-bin minima (earlier position on ties), then
    the k smallest (value, position) pairs of the minima."""
    values = np.asarray(values, dtype=np.int64)
    ids = np.asarray(ids)
    n = len(values)
    b = bin_of(n, l)
    starts = np.searchsorted(b, np.arange(l), side="left")
    ends = np.searchsorted(b, np.arange(l), side="right")
    mval, mpos = [], []
    for i in range(l):
        seg = values[starts[i]:ends[i]]
        r = int(np.argmin(seg))
        mval.append(int(seg[r]))
        mpos.append(int(starts[i] + r))
    order = np.lexsort((np.array(mpos), np.array(mval)))[:k]
    return [mval[o] for o in order], [int(ids[mpos[o]]) for o in order]


def expected_hits(n: int, k: int, l: int) -> float:
    """E|I| for ApproxTopk: each of the true k smallest is found iff it is the
    smallest true-top-k element of its bin, so E|I| = number of bins that hold
    at least one of the k.  With random positions and bins of sizes s_i,
    Pr[bin i empty of them] = C(n - s_i, k) / C(n, k)."""
    sizes = np.bincount(bin_of(n, l), minlength=l)
    tot = 0.0
    logc = math.lgamma(n + 1) - math.lgamma(k + 1) - math.lgamma(n - k + 1)
    for s in np.unique(sizes):
        cnt = int(np.sum(sizes == s))
        if n - s >= k:
            le = (math.lgamma(n - s + 1) - math.lgamma(k + 1)
                  - math.lgamma(n - s - k + 1)) - logc
            p_empty = math.exp(le)
        else:
            p_empty = 0.0
        tot += cnt * (1.0 - p_empty)
    return tot
