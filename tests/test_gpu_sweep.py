"""Angle sweeps of the amplitude (qt_contract_sweep): several (gamma, beta) sets contracted
with one order, slicing and schedule. Each set's amplitude matches the FP64 oracle built
with that set's angles, and equals, bit for bit, a qt_contract call at those angles."""

import pytest

from helpers import oracle_amplitude, oracle_plan, oracle_problem, rel_err
from oracle import network
from paper_2012_02430_gb300.inputs import random_angles

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [(24, 2, 3, 0, 5), (40, 2, 11, -4, 6), (30, 3, 7, -2, 4), (80, 2, 1002, 26 - 35, 3)]


@pytest.mark.parametrize("case", CASES)
def test_amplitude_sweep_matches_oracle(qt, case):
    n, p, seed, off, n_sets = case
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    sets = [random_angles(p, 7000 + s) for s in range(n_sets)]
    gs = [list(g) for g, _ in sets]
    bs = [list(b) for _, b in sets]
    net = qt.Network(edges, n, p, gammas, betas, z)
    w = net.order(0)
    if off:
        net.slice(w + off, 6, 1)
    net.prepare(0, batch=2)
    amps = net.contract_sweep(gs, bs)
    assert len(amps) == n_sets
    plan = oracle_plan(adj, 0, w + off, 6, 1) if off else oracle_plan(adj, 0)
    for s in range(n_sets):
        t_s, _, norm_s = network.build_network(n, edges, p, gs[s], bs[s], z)
        ref, _ = oracle_amplitude(t_s, norm_s, plan)
        assert rel_err(amps[s], ref) <= 1e-5, (s, amps[s], ref)
        qt.qt_set_angles(net.handle, gs[s], bs[s])
        single = net.contract(0)
        assert single == amps[s], (s, single, amps[s])
