"""Oracle: step-dependent slicing (Sec. VI.C late parallelisation, Sec. VI.D, Fig. 8, Alg. 1).

TEST INFRASTRUCTURE (see oracle/network.py).

Slicing a vertex fixes the value of its index: the vertex leaves the graph
without joining its neighbours, and the expression splits into 2 parts whose
sum is the original (Eq. 2). The search, per round:
  1. order the current graph greedily and find its peak, the first step with the
     largest neighbour count;
  2. for every step s from 0 up to the peak: eliminate the first s vertices of
     that order, then remove r vertices one at a time, each time the one with
     the most neighbours at that moment (ties: smaller id), and order the rest
     greedily again;
  3. keep the s whose plan has the smallest width, then the smallest sum of
     2^w over its steps (summed in step order in double precision), then the
     smallest s; its first s eliminations and its r vertices join the schedule.
Rounds repeat while the width exceeds width_limit and fewer than max_vars
vertices are sliced; the last round takes min(r, max_vars - sliced) vertices.
The widths counted are those of every step of the plan: the steps fixed by
earlier rounds, the first s steps of this round and the new greedy order.

Execution reading (the paper is silent on it for several rounds): every slice
id fixes all k sliced indices right after the first round's step s_1; steps
before s_1 run once on the unsliced network, steps from s_1 on run per slice.
"""

from __future__ import annotations

import math

import numpy as np

from .ordering import MIN_FILL, eliminate, greedy_order, remove_vertex


def _plan_cost(widths):
    total = 0.0
    for w in widths:
        total += math.ldexp(1.0, int(w))
    return total


def step_dependent_slicing(adj: np.ndarray, algo: int = MIN_FILL, width_limit: int = 1 << 30,
                           max_vars: int = 0, r: int = 1, keep=None):
    """Returns a dict with the schedule: order, sliced, slice_step, rounds, width, widths.
    Vertices in `keep` (open indices) are never eliminated nor sliced."""
    if width_limit < 1 or r < 1 or max_vars < 0:
        raise ValueError("bad slicing parameters")
    a = adj.copy()
    np.fill_diagonal(a, False)
    n = a.shape[0]
    alive = np.ones(n, dtype=bool)
    keep = np.zeros(n, dtype=bool) if keep is None else np.asarray(keep, dtype=bool)
    order, widths = greedy_order(a, alive, algo, keep)
    done_order, done_widths = [], []
    sliced, rounds = [], []
    width = max(widths, default=0)
    while width > width_limit and len(sliced) < max_vars and (alive & ~keep).any():
        rr = min(r, max_vars - len(sliced))
        peak = int(np.argmax(widths))
        best = None
        for s in range(peak + 1):
            b = a.copy()
            al = alive.copy()
            for v in order[:s]:
                eliminate(b, al, v)
            removed = []
            for _ in range(rr):
                ids = np.flatnonzero(al & ~keep)
                if len(ids) == 0:
                    break
                deg = b[ids].sum(axis=1)
                v = int(ids[np.lexsort((ids, -deg))[0]])
                remove_vertex(b, al, v)
                removed.append(v)
            o2, w2 = greedy_order(b, al, algo, keep)
            plan_w = done_widths + widths[:s] + w2
            key = (max(plan_w, default=0), _plan_cost(plan_w), s)
            if best is None or key < best[0]:
                best = (key, s, removed, o2, w2, b, al)
        key, s, removed, o2, w2, b, al = best
        rounds.append((len(done_order) + s, list(removed)))
        done_order += order[:s]
        done_widths += widths[:s]
        sliced += removed
        a, alive = b, al
        order, widths = o2, w2
        width = key[0]
    full_order = done_order + order
    return {
        "order": full_order,
        "sliced": sliced,
        "slice_step": rounds[0][0] if rounds else 0,
        "rounds": rounds,
        "width": max(done_widths + widths, default=0),
        "widths": done_widths + widths,
    }
