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


def oracle_plan(adj, algo=0, width_limit=1 << 30, max_vars=0, r=1):
    return slicing.step_dependent_slicing(adj, ALGO[algo], width_limit, max_vars, r)


def oracle_amplitude(tensors, norm, plan, slice_ids=None):
    total, per = contract.contract_amplitude(tensors, plan["order"], plan["sliced"],
                                             plan["slice_step"], slice_ids)
    return total * norm, [x * norm for x in per]


def rel_err(a, b):
    return abs(a - b) / abs(b)
