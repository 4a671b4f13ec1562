"""Shared test helpers: oracle plans/amplitudes and GPU runs through the C ABI."""

from __future__ import annotations

from oracle import contract, network, ordering, slicing
from paper_2012_02430_gb300.inputs import qaoa_instance

ALGO = {0: ordering.MIN_FILL, 1: ordering.MIN_DEGREE}


def oracle_problem(n, p, seed):
    edges, gammas, betas, z = qaoa_instance(n, p, seed)
    tensors, nv, norm = network.build_network(n, edges, p, gammas, betas, z)
    adj = ordering.adjacency_matrix(network.line_graph(tensors, nv), nv)
    return edges, gammas, betas, z, tensors, nv, norm, adj


def oracle_problem_open(n, p, seed, opens):
    """As oracle_problem with the qubits `opens` left open (Sec. VII); also returns the
    open variables and the keep mask of the planner."""
    import numpy as np
    edges, gammas, betas, z = qaoa_instance(n, p, seed)
    tensors, nv, norm = network.build_network(n, edges, p, gammas, betas, z, opens)
    sets = network.open_clique(network.line_graph(tensors, nv), n, p, len(opens))
    adj = ordering.adjacency_matrix(sets, nv)
    keep = np.zeros(nv, dtype=bool)
    keep[n * p:] = True
    open_vars = list(range(n * p, nv))
    return edges, gammas, betas, z, tensors, nv, norm, adj, keep, open_vars


def oracle_plan(adj, algo=0, width_limit=1 << 30, max_vars=0, r=1, keep=None):
    return slicing.step_dependent_slicing(adj, ALGO[algo], width_limit, max_vars, r, keep)


def oracle_amplitude(tensors, norm, plan, slice_ids=None, open_vars=()):
    total, per = contract.contract_amplitude(tensors, plan["order"], plan["sliced"],
                                             plan["slice_step"], slice_ids, open_vars)
    return total * norm, [x * norm for x in per]


def batch_vector(t, a):
    """Flattens an oracle result tensor over a open variables to the library's order:
    entry b has bit j = the value of open variable j."""
    import numpy as np
    t = np.asarray(t)
    return np.array([t[tuple((b >> j) & 1 for j in range(a))] for b in range(1 << a)])


def rel_err(a, b):
    return abs(a - b) / abs(b)
