"""Oracle: candidates, features and labels of the learned slicing proposals.

TEST INFRASTRUCTURE (see oracle/network.py).

One slicing round (Sec. VI.C-D) on the greedy order of the current graph: a
candidate is (s, v) with s from 0 to the first peak and v among the `topv`
alive vertices of largest degree after the first s eliminations (ties: smaller
id; rank j). Its 16 features, with W the peak width, peak the peak position,
deg the degree after s eliminations, A the alive count, E the edge count:
  0 s/(peak+1)   1 w[s]/W   2 deg(v)/W   3 max deg/W   4 j/topv   5 A/n0
  6 (2E/A)/W   7 max(w[:s])/W (0 if s=0)   8 log2(1 + sum_{i<s} 2^w[i])/W
  9 fill(v)/max(1, deg(v)(deg(v)-1)/2)   10 #{deg = max deg}/A
  11 deg(peak vertex)/W (0 if eliminated)   12 v is the peak vertex or adjacent to it
  13 (peak-s)/(peak+1)   14 w[s-1]/W (0 if s=0)   15 E/max(1, A(A-1)/2)
Its label is the width of the plan that eliminates the first s vertices, slices v
and re-orders the rest greedily, divided by W.
"""

from __future__ import annotations

import math

import numpy as np

from .ordering import eliminate, greedy_order, remove_vertex


def round_candidates(adj, order, widths, n0, topv):
    peak = int(np.argmax(widths))
    W = max(1, widths[peak])
    a = adj.copy()
    np.fill_diagonal(a, False)
    alive = np.ones(a.shape[0], dtype=bool)
    pv = order[peak]
    out = []
    prefix_cost = 0.0
    prefix_max = 0
    for s in range(peak + 1):
        if s > 0:
            eliminate(a, alive, order[s - 1])
            prefix_cost += math.ldexp(1.0, int(widths[s - 1]))
            prefix_max = max(prefix_max, int(widths[s - 1]))
        ids = np.flatnonzero(alive)
        if len(ids) == 0:
            break
        deg = a[ids].sum(axis=1)
        ranked = [int(ids[i]) for i in np.lexsort((ids, -deg))]
        dmax = int(deg.max())
        A = len(ids)
        E = deg.sum() / 2.0
        nmax = int((deg == dmax).sum())
        dpeak = int(a[pv].sum()) if alive[pv] else 0
        for j, v in enumerate(ranked[:topv]):
            nb = np.flatnonzero(a[v])
            dv = len(nb)
            present = int(a[np.ix_(nb, nb)].sum()) // 2
            fill = dv * (dv - 1) // 2 - present
            near = v == pv or (alive[pv] and a[v, pv])
            f = [s / (peak + 1), widths[s] / W, dv / W, dmax / W, j / topv, A / n0,
                 (2.0 * E / A) / W, prefix_max / W, math.log2(1.0 + prefix_cost) / W,
                 fill / max(1.0, dv * (dv - 1) / 2.0), nmax / A, dpeak / W, 1.0 if near else 0.0,
                 (peak - s) / (peak + 1), (widths[s - 1] / W) if s > 0 else 0.0,
                 E / max(1.0, A * (A - 1) / 2.0)]
            out.append((s, v, j, f))
    return out


def candidate_width(adj, order, widths, s, v, algo):
    a = adj.copy()
    np.fill_diagonal(a, False)
    alive = np.ones(a.shape[0], dtype=bool)
    for x in order[:s]:
        eliminate(a, alive, x)
    remove_vertex(a, alive, v)
    _, w2 = greedy_order(a, alive, algo)
    return max(list(widths[:s]) + list(w2) + [0])


def dataset(adj, algo, topv):
    """(features, labels, meta) of every candidate of the first round."""
    order, widths = greedy_order(adj, None, algo)
    W = max(1, max(widths))
    feats, labels, meta = [], [], []
    for s, v, j, f in round_candidates(adj, order, widths, adj.shape[0], topv):
        w = candidate_width(adj, order, widths, s, v, algo)
        feats.append(f)
        labels.append(w / W)
        meta.append((s, v, w))
    return np.array(feats), np.array(labels), meta
