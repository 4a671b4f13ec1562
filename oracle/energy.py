"""Oracle: MaxCut energy <C> from per-edge lightcone networks (Sec. III.A-B), FP64.

TEST INFRASTRUCTURE (see oracle/network.py).

The energy <gamma beta| C |gamma beta> is a duplicated (bra-ket) tensor
expression with the observable in the middle (Sec. III.B). Per edge (u, v) only
the gates in the backward lightcone of Z_u Z_v survive (the lightcone remark of
Sec. III.A): with d(w) the graph distance from w to {u, v}, the layer-k cost
gate on edge (a, b) stays iff min(d(a), d(b)) <= p - k, the layer-k mixer on w
stays iff d(w) <= p - k, and |+> stays on every w with d(w) <= p.

Network of one edge: qubit w with L(w) = max(0, p - d(w)) mixers has ket
variables (w, 0..L(w)-1), bra variables likewise, and one final variable shared
by ket and bra (the trace over the output). Ket gates act on ket variables, bra
gates are their complex conjugates on bra variables, and the observable is the
vector (1, -1) on the final variable of u and of v. <Z_u Z_v> is 2^(-|S|) times
the full contraction, S the set of qubits with d(w) <= p.
"""

from __future__ import annotations

import math
from collections import deque

import numpy as np

from .contract import contract_amplitude
from .network import line_graph, mixer_matrix, phase_matrix
from .ordering import MIN_FILL, adjacency_matrix, greedy_order


def distances_to_edge(n, edges, u, v):
    nb = [[] for _ in range(n)]
    for (a, b) in edges:
        nb[a].append(b)
        nb[b].append(a)
    d = [-1] * n
    q = deque()
    for s in (u, v):
        d[s] = 0
        q.append(s)
    while q:
        a = q.popleft()
        for b in nb[a]:
            if d[b] < 0:
                d[b] = d[a] + 1
                q.append(b)
    return d


def lightcone_network(n, edges, p, gammas, betas, u, v):
    """Tensors of the bra-ket network for <Z_u Z_v>; returns (tensors, n_vars, norm)."""
    d = distances_to_edge(n, edges, u, v)
    qubits = [w for w in range(n) if 0 <= d[w] <= p]
    nmix = {w: max(0, p - d[w]) for w in qubits}
    ids = {}

    def var(key):
        return ids.setdefault(key, len(ids))

    def ket(w, t):
        return var(("f", w)) if t >= nmix[w] else var(("k", w, t))

    def bra(w, t):
        return var(("f", w)) if t >= nmix[w] else var(("b", w, t))

    tensors = []
    plus = np.array([1.0, 1.0], dtype=np.complex128)
    for side, idx, conj in (("ket", ket, False), ("bra", bra, True)):
        for w in qubits:
            tensors.append(((idx(w, 0),), plus.copy()))
        for k in range(1, p + 1):
            dm = phase_matrix(gammas[k - 1])
            mm = mixer_matrix(betas[k - 1])
            if conj:
                dm, mm = dm.conj(), mm.conj()
            for (a, b) in edges:
                if d[a] >= 0 and d[b] >= 0 and min(d[a], d[b]) <= p - k:
                    tensors.append(((idx(a, k - 1), idx(b, k - 1)), dm.copy()))
            for w in qubits:
                if d[w] <= p - k:
                    tensors.append(((idx(w, k - 1), idx(w, k)), mm.copy()))
    z = np.array([1.0, -1.0], dtype=np.complex128)
    tensors.append(((var(("f", u)),), z.copy()))
    tensors.append(((var(("f", v)),), z.copy()))
    return tensors, len(ids), 2.0 ** (-len(qubits))


def zz_lightcone(n, edges, p, gammas, betas, u, v, algo=MIN_FILL):
    tensors, nv, norm = lightcone_network(n, edges, p, gammas, betas, u, v)
    adj = adjacency_matrix(line_graph(tensors, nv), nv)
    order, _ = greedy_order(adj, None, algo)
    total, _ = contract_amplitude(tensors, order)
    return norm * total


def energy_lightcone(n, edges, p, gammas, betas):
    """(energy, per-edge <Z_u Z_v>) with every edge contracted on its lightcone."""
    zz = [zz_lightcone(n, edges, p, gammas, betas, u, v).real for (u, v) in edges]
    return sum(0.5 * (1.0 - x) for x in zz), zz


def edge_energy_p1_closed_form(n, edges, gamma, beta, u, v):
    """<(1 - Z_u Z_v)/2> at p = 1 for any graph (Wang, Hadfield, Jiang, Rieffel 2018).

    With degrees d_u, d_v and lam = number of triangles containing (u, v):
    1/2 + 1/4 sin(4b) sin(g) (cos^(d_u-1) g + cos^(d_v-1) g)
        - 1/4 sin^2(2b) cos^(d_u+d_v-2-2 lam) g (1 - cos^lam (2g)).
    """
    nb = [set() for _ in range(n)]
    for (a, b) in edges:
        nb[a].add(b)
        nb[b].add(a)
    du, dv = len(nb[u]) - 1, len(nb[v]) - 1
    lam = len((nb[u] - {v}) & (nb[v] - {u}))
    g, b = gamma, beta
    term1 = 0.25 * math.sin(4 * b) * math.sin(g) * (math.cos(g) ** du + math.cos(g) ** dv)
    term2 = 0.25 * math.sin(2 * b) ** 2 * math.cos(g) ** (du + dv - 2 * lam) * (1 - math.cos(2 * g) ** lam)
    return 0.5 + term1 - term2
