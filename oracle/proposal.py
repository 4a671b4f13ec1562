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

from .ordering import MIN_FILL, eliminate, greedy_order, remove_vertex


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


# ----------------------------------------------------------------------------
# Learned elimination steps. At a step of a greedy ordering, the candidates are
# the topc alive vertices best by the greedy key (min-fill: fill, degree, id;
# min-degree: degree, id). Features of candidate j (W0 = the greedy width of
# the whole graph, n0 = its vertex count, maxw = largest width taken so far,
# A alive vertices, E edges, dmax the largest degree, c0 = rank-0 candidate):
#   0 deg/W0   1 fill/max(1, deg(deg-1)/2)   2 j/#candidates
#   3 (fill - fill(c0))/W0   4 (deg - deg(c0))/W0   5 mean neighbour degree/W0
#   6 max neighbour degree/W0   7 min neighbour degree/W0 (0 without neighbours)
#   8 A/n0   9 t/n0   10 maxw/W0   11 (2E/A)/W0   12 E/max(1, A(A-1)/2)
#   13 1 for j = 0, else |N(v) & N(c0)|/max(1, deg)   14 deg/max(1, dmax)
#   15 |N(v) | N(N(v))|/max(1, A)
# Label: log2 of sum 2^w over the order "greedy steps so far, the candidate,
# greedy after".
# ----------------------------------------------------------------------------

def _fill(a, v):
    nb = np.flatnonzero(a[v])
    d = len(nb)
    present = int(a[np.ix_(nb, nb)].sum()) // 2
    return d * (d - 1) // 2 - present


def step_candidates(a, alive, topc, algo):
    ids = np.flatnonzero(alive)
    keys = []
    for v in ids:
        d = int(a[v].sum())
        f = _fill(a, v) if algo == MIN_FILL else 0
        keys.append((f, d, int(v)))
    keys.sort()
    return [(v, d, f) for f, d, v in keys[:topc]]


def step_features(a, alive, cands, j, t, n0, W0, maxw):
    W = max(1, W0)
    v, deg, fill = cands[j]
    ids = np.flatnonzero(alive)
    A = len(ids)
    degs = a[ids].sum(axis=1)
    E = degs.sum() / 2.0
    dmax = int(degs.max()) if A else 0
    nb = np.flatnonzero(a[v])
    nd = a[nb].sum(axis=1) if len(nb) else np.array([0])
    two = a[nb].any(axis=0) | a[v] if len(nb) else a[v].copy()
    v0, deg0, fill0 = cands[0]
    common = int((a[v] & a[v0]).sum())
    return [deg / W, fill / max(1.0, deg * (deg - 1) / 2.0), j / max(1, len(cands)),
            (fill - fill0) / W, (deg - deg0) / W,
            (nd.sum() / deg) / W if deg else 0.0, (nd.max() / W) if deg else 0.0,
            (nd.min() / W) if deg else 0.0, A / n0, t / n0, maxw / W,
            ((2.0 * E / A) if A else 0.0) / W, E / max(1.0, A * (A - 1) / 2.0),
            1.0 if j == 0 else common / max(1.0, deg), deg / max(1.0, dmax),
            int(two.sum()) / max(1.0, A)]


def order_dataset(adj, algo, topc, stride):
    """(features, labels, meta) of the candidates at every stride-th step of the greedy
    order of adj."""
    order, widths = greedy_order(adj, None, algo)
    W0 = max(widths, default=0)
    n0 = adj.shape[0]
    a = adj.copy()
    np.fill_diagonal(a, False)
    alive = np.ones(n0, dtype=bool)
    feats, labels, meta = [], [], []
    prefix, maxw = [], 0
    for t, x in enumerate(order):
        if t % stride == 0:
            cands = step_candidates(a, alive, topc, algo)
            if len(cands) >= 2:
                for j, (v, deg, fill) in enumerate(cands):
                    feats.append(step_features(a, alive, cands, j, t, n0, W0, maxw))
                    b = a.copy()
                    al = alive.copy()
                    d = int(b[v].sum())
                    eliminate(b, al, v)
                    _, rest = greedy_order(b, al, algo)
                    ws = prefix + [d] + list(rest)
                    labels.append(math.log2(max(1.0, sum(math.ldexp(1.0, int(w)) for w in ws))))
                    meta.append((t, v, max(ws)))
        prefix.append(int(widths[t]))
        maxw = max(maxw, int(widths[t]))
        eliminate(a, alive, x)
    return np.array(feats), np.array(labels), meta
