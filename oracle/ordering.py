"""Oracle: greedy elimination orders and the contraction width (Sec. IV.B, Sec. V.A.1).

TEST INFRASTRUCTURE (see oracle/network.py).

Eliminating a vertex v deletes it and joins all of its neighbours into a
clique; the result tensor of that step has rank N_G(v), the number of v's
neighbours at that moment. The contraction width is c = max over steps of that
count (Sec. IV.B, the cost formula C ~ 2^c).

Two greedy rules, each a deterministic argmin over the remaining vertices:
  * min-degree (Sec. V.A.1, "contracts the lowest-degree vertex"): key (deg, id);
  * min-fill (the default): key (fill, deg, id), where fill(v) is the number of
    pairs of v's neighbours that are not yet adjacent.
Ties go to the smaller vertex id (the paper states no tie-break).
"""

from __future__ import annotations

import numpy as np

MIN_FILL = 0
MIN_DEGREE = 1


def adjacency_matrix(adj_sets, n_vars):
    a = np.zeros((n_vars, n_vars), dtype=bool)
    for v, nb in enumerate(adj_sets):
        for w in nb:
            a[v, w] = True
    return a


def greedy_order(adj: np.ndarray, alive=None, algo: int = MIN_FILL, keep=None):
    """Greedy order of the alive vertices of the symmetric boolean matrix adj.

    Returns (order, widths): widths[i] is the neighbour count of order[i] when it
    is eliminated. adj is not modified. Vertices marked in `keep` (open indices of
    a batch of amplitudes) stay in the graph and are never eliminated.
    """
    a = adj.copy()
    n = a.shape[0]
    alive = np.ones(n, dtype=bool) if alive is None else alive.copy()
    keep = np.zeros(n, dtype=bool) if keep is None else np.asarray(keep, dtype=bool)
    np.fill_diagonal(a, False)
    a[~alive, :] = False
    a[:, ~alive] = False
    order, widths = [], []
    while (alive & ~keep).any():
        ids = np.flatnonzero(alive)
        sub = a[np.ix_(ids, ids)]
        deg = sub.sum(axis=1).astype(np.int64)
        if algo == MIN_FILL:
            f = sub.astype(np.float64)
            # edges among the neighbours of each vertex = row sums of (A @ A) * A / 2
            tri = ((f @ f) * f).sum(axis=1)
            fill = deg * (deg - 1) // 2 - np.rint(tri / 2).astype(np.int64)
            key = np.lexsort((ids, deg, fill))
        elif algo == MIN_DEGREE:
            key = np.lexsort((ids, deg))
        else:
            raise ValueError("unknown ordering algorithm")
        key = [i for i in key if not keep[ids[i]]]
        v = int(ids[key[0]])
        nb = np.flatnonzero(a[v])
        order.append(v)
        widths.append(len(nb))
        eliminate(a, alive, v, nb)
    return order, widths


def eliminate(a: np.ndarray, alive: np.ndarray, v: int, nb=None):
    """Remove vertex v after joining its neighbours into a clique (in place)."""
    if nb is None:
        nb = np.flatnonzero(a[v])
    a[np.ix_(nb, nb)] = True
    a[nb, nb] = False
    a[v, :] = False
    a[:, v] = False
    alive[v] = False


def remove_vertex(a: np.ndarray, alive: np.ndarray, v: int):
    """Slice a vertex away: delete it without joining its neighbours."""
    a[v, :] = False
    a[:, v] = False
    alive[v] = False


def replay_widths(adj: np.ndarray, order, alive=None):
    """Neighbour counts along a given order (no choice made): the width profile."""
    a = adj.copy()
    n = a.shape[0]
    alive = np.ones(n, dtype=bool) if alive is None else alive.copy()
    np.fill_diagonal(a, False)
    a[~alive, :] = False
    a[:, ~alive] = False
    widths = []
    for v in order:
        nb = np.flatnonzero(a[v])
        widths.append(len(nb))
        eliminate(a, alive, v, nb)
    return widths
