"""Oracle: the randomised greedy ordering "rgreedy" (Sec. V.A.2).

TEST INFRASTRUCTURE (see oracle/network.py).

Instead of always eliminating a vertex of smallest degree, every step draws the
next vertex v with probability proportional to the Boltzmann weight
exp(-N_G(v) / tau), N_G(v) being v's current neighbour count; the whole
elimination is repeated q times and the best of the q orders is kept.

Readings (the paper gives only the weight and "best of q"):
  * best = smallest width, then smallest sum of 2^w over the steps (in step order,
    double precision), then the earliest run;
  * the weights are shifted by the smallest degree of the step, w(v) =
    r^(N_G(v) - d_min) with r = exp(-1/tau) computed once and the power taken by
    repeated multiplication: the same distribution, no overflow for small tau;
  * one draw per step: u uniform in [0, 1), target = u * (sum of the weights in
    ascending vertex id); the vertex taken is the first whose running sum exceeds
    the target (the last candidate if rounding leaves none);
  * the draws come from one SplitMix64 stream (Steele, Lea, Flood, OOPSLA 2014)
    seeded with `seed`, consumed run after run, u = (x >> 11) * 2^-53. This file
    implements the generator itself from that definition.
Kept vertices (open indices) are never eliminated, as in ordering.greedy_order.
"""

from __future__ import annotations

import math

import numpy as np

from .ordering import eliminate

_MASK64 = (1 << 64) - 1


class _SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def uniform(self) -> float:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        z ^= z >> 31
        return (z >> 11) * (1.0 / (1 << 53))


def boltzmann_weights(degrees, tau: float):
    """w(v) proportional to exp(-deg(v)/tau), shifted by the smallest degree."""
    r = math.exp(-1.0 / tau)
    dmin = min(degrees)
    out = []
    for d in degrees:
        w = 1.0
        for _ in range(d - dmin):
            w *= r
        out.append(w)
    return out


def rgreedy_run(adj: np.ndarray, tau: float, rng: _SplitMix64, keep=None):
    """One randomised elimination: returns (order, widths)."""
    a = adj.copy()
    n = a.shape[0]
    np.fill_diagonal(a, False)
    alive = np.ones(n, dtype=bool)
    keep = np.zeros(n, dtype=bool) if keep is None else np.asarray(keep, dtype=bool)
    order, widths = [], []
    while (alive & ~keep).any():
        cand = [int(v) for v in np.flatnonzero(alive & ~keep)]
        deg = [int(a[v].sum()) for v in cand]
        w = boltzmann_weights(deg, tau)
        total = 0.0
        for x in w:
            total += x
        target = rng.uniform() * total
        pick = cand[-1]
        run = 0.0
        for v, x in zip(cand, w):
            run += x
            if run > target:
                pick = v
                break
        nb = np.flatnonzero(a[pick])
        order.append(pick)
        widths.append(len(nb))
        eliminate(a, alive, pick, nb)
    return order, widths


def rgreedy_order(adj: np.ndarray, tau: float, q: int, seed: int, keep=None):
    """Best of q randomised eliminations. Returns (order, widths, run_widths)."""
    if tau <= 0 or q < 1:
        raise ValueError("need tau > 0 and q >= 1")
    rng = _SplitMix64(seed)
    best = None
    run_widths = []
    for run in range(q):
        o, w = rgreedy_run(adj, tau, rng, keep)
        cost = 0.0
        for x in w:
            cost += math.ldexp(1.0, x)
        key = (max(w, default=0), cost, run)
        run_widths.append(key[0])
        if best is None or key < best[0]:
            best = (key, o, w)
    return best[1], best[2], run_widths
