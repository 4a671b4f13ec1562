"""The tiled GEMM's tensor-copy (TMA) staging against the FP64 oracle: the same
amplitudes, bit for bit, as the cp.async staging, no bounded wait giving up, and
the tensor-copy kernel really launched."""

import pytest

from helpers import oracle_amplitude, oracle_plan, oracle_problem, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", [(44, 2, 14, -4), (60, 2, 18, -4), (80, 2, 1002, 26 - 35)])
def test_tma_staging_matches_oracle(qt, case):
    n, p, seed, off = case
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    amps = {}
    for tma in (0, 1):
        net = qt.Network(edges, n, p, gammas, betas, z)
        qt.qt_set_option(net.handle, qt.QT_OPT_GEMM, 1)
        qt.qt_set_option(net.handle, qt.QT_OPT_TMA, tma)
        w = net.order(0)
        net.slice(w + off, 6, 1)
        net.prepare(0, batch=4)
        amps[tma] = net.contract(0)  # raises QT_ETIMEOUT if a bounded wait gave up
        st = net.stats()
        assert st["gemm_groups"] > 0
        assert (st["tma_gemm_launches"] > 0) == bool(tma), st["tma_gemm_launches"]
    plan = oracle_plan(adj, 0, w + off, 6, 1)
    ref, _ = oracle_amplitude(tensors, norm, plan)
    for tma in (0, 1):
        assert rel_err(amps[tma], ref) <= 1e-5, (tma, amps[tma], ref)
    assert abs(amps[0] - amps[1]) <= 1e-12 * abs(ref)
