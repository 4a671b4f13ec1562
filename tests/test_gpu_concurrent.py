"""Slice-phase launches run on several streams inside the captured graph (QT_OPT_CONCURRENT):
with the same kernel choices, the same amplitudes, bit for bit, as on one stream, and within
the complex64 bar of the FP64 oracle, over sliced and unsliced plans, several batches, and
the bench workload."""

import pytest

from helpers import oracle_amplitude, oracle_plan, oracle_problem, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [(30, 2, 5, 0, 1), (44, 2, 14, -4, 3), (60, 2, 18, -4, 4), (50, 3, 1003, -4, 2),
         (80, 2, 1002, 26 - 35, 4)]


@pytest.mark.parametrize("case", CASES)
def test_concurrent_graph_matches_serial(qt, case):
    n, p, seed, off, batch = case
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    amps = {}
    for conc in (0, 1):
        net = qt.Network(edges, n, p, gammas, betas, z)
        qt.qt_set_option(net.handle, qt.QT_OPT_CONCURRENT, conc)
        w = net.order(0)
        if off:
            net.slice(w + off, 6, 1)
        net.prepare(0, batch=batch)  # default kernels (no autotuning): the same choices
        first = net.contract(0)
        again = net.contract(0)  # the captured graph replayed
        assert first == again
        amps[conc] = first
    assert amps[0] == amps[1], amps
    plan = oracle_plan(adj, 0, w + off, 6, 1) if off else oracle_plan(adj, 0)
    ref, _ = oracle_amplitude(tensors, norm, plan)
    assert rel_err(amps[1], ref) <= 1e-5, (amps[1], ref)
