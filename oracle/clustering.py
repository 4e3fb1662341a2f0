"""Algorithm 4 (ClusteringKNNS, plaintext clustering-based k-NNS) written out,
on a server layout given as input.

TEST INFRASTRUCTURE ONLY (the oracle): only tests/, __graft_entry__.smoke()
and bench.py's cpu_baseline and reference legs may import this module.  It never imports the
CUDA package.

The server's layout is what Algorithm 4 receives: T groups of clusters with
their centres (the centres of a group already in the server's random order,
so a centre is named by its position), the clusters' members, and the stash
in the server's random order.  Steps, in the paper's order:

  for every group i: d_j = |q - c_j|^2 for every centre, truncated
      d_j >> r_c; u^i centres by ApproxTopk over l^i bins (Algorithm 2), or
      exactly when l^i = 0;
  C = the union of the selected clusters, in the order the selections list
      them (group by group, each group's picks smallest first);
  for every point of C and of the stash S: |q - p|^2 >> r_p;
  k candidates from C by exact selection (NaiveTopk, Algorithm 1) and k from
      S by ApproxTopk over l_s bins;
  the final k of the 2k candidates by exact selection (those from C first).

Ties are broken by position everywhere (the (value, position) reading of
Algorithms 1 and 2 in select.py).  Fewer than k points in C or S leave
(MAXVAL, -1) candidates, MAXVAL = t - 1, above every distance.
"""
from __future__ import annotations

import numpy as np

from . import select


def sq_dist(points: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Exact squared Euclidean distances of integer points to q."""
    diff = points.astype(np.int64) - q.astype(np.int64)[None, :]
    return np.sum(diff * diff, axis=1)


def _select(values: np.ndarray, ids: np.ndarray, k: int, bins: int):
    if bins:
        return select.approx_topk_by_position(values, ids, k, bins)
    return select.exact_topk(values, ids, k)


def clustering_knns(q: np.ndarray, coords: np.ndarray, group_offsets, centre_cluster,
                    centres: np.ndarray, cl_offsets, cl_members, stash: np.ndarray,
                    k: int, u, l, l_s: int, r_c: int, r_p: int, maxval: int):
    """Returns the k ids (numpy int64) Algorithm 4 outputs for query q.

    group_offsets [T + 1]: group i's centres sit at positions
    group_offsets[i] .. group_offsets[i+1] of `centres` (uint8 [.][d]);
    centre_cluster[pos] is the cluster id of the centre at position pos;
    cluster c's points are cl_members[cl_offsets[c]:cl_offsets[c+1]];
    stash[x] is the point id at stash position x."""
    T = len(group_offsets) - 1
    picked = []
    for i in range(T):
        g0, g1 = int(group_offsets[i]), int(group_offsets[i + 1])
        dc = sq_dist(centres[g0:g1], q) >> r_c
        ui = min(int(u[i]), g1 - g0)
        li = max(min(int(l[i]), g1 - g0), ui) if l[i] else 0
        _, pos = _select(dc, np.arange(g1 - g0), ui, li)
        picked += [int(centre_cluster[g0 + p]) for p in pos]
    C = np.concatenate([cl_members[int(cl_offsets[c]):int(cl_offsets[c + 1])] for c in picked]
                       + [np.zeros(0, dtype=np.int64)]).astype(np.int64)
    cand_v = [maxval] * (2 * k)
    cand_i = [-1] * (2 * k)
    if len(C):
        dv = sq_dist(coords[C], q) >> r_p
        v, i = select.exact_topk(dv, C, min(k, len(C)))
        cand_v[:len(v)], cand_i[:len(i)] = v, i
    if len(stash):
        ds = sq_dist(coords[stash], q) >> r_p
        ks = min(k, len(stash))
        ls = max(min(l_s, len(stash)), ks) if l_s else 0
        v, i = _select(ds, stash.astype(np.int64), ks, ls)
        cand_v[k:k + len(v)], cand_i[k:k + len(i)] = v, i
    _, fin = select.exact_topk(np.array(cand_v), np.array(cand_i), k)
    return np.array(fin, dtype=np.int64)
