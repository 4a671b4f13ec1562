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


# the last four reach the tensor-copy kernel's four ways of pairing summed values:
# A over k or x, B over k or y
TRI_CASES = [(36, 2, 7, 0, 1), (30, 3, 7, -2, 2), (50, 2, 2, -4, 3), (56, 2, 4, -2, 2),
             (44, 3, 1, -2, 1), (80, 2, 1002, 26 - 35, 4), (24, 3, 35, -2, 2),
             (30, 3, 19, 0, 2), (32, 2, 2, 0, 2), (32, 3, 25, 0, 2)]


@pytest.mark.parametrize("case", TRI_CASES)
def test_tma_triangle_matches_oracle(qt, case):
    """Triangle-form launches with tensor-copy staging (the default, its own tiles of
    2^7..2^9 outputs) and with the cp.async kernel: both within the complex64 bar of the
    oracle, and every case's triangle launch really takes the tensor-copy kernel."""
    n, p, seed, off, batch = case
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    amps, launches = {}, {}
    for tma in (0, 1):
        net = qt.Network(edges, n, p, gammas, betas, z)
        qt.qt_set_option(net.handle, qt.QT_OPT_TRIANGLE, 1)
        qt.qt_set_option(net.handle, qt.QT_OPT_TMA, tma)
        w = net.order(0)
        if off:
            net.slice(w + off, 6, 1)
        net.prepare(0, batch=batch)
        amps[tma] = net.contract(0)
        st = net.stats()
        assert st["tri_groups"] >= 1
        launches[tma] = st["tma_gemm_launches"]
    plan = oracle_plan(adj, 0, w + off, 6, 1) if off else oracle_plan(adj, 0)
    ref, _ = oracle_amplitude(tensors, norm, plan)
    for tma in (0, 1):
        assert rel_err(amps[tma], ref) <= 1e-5, (tma, amps[tma], ref)
    assert launches[0] == 0
    assert launches[1] > 0  # every case's triangle launch takes the tensor-copy kernel


BLOCK_CASES = [(44, 2, 14, -4), (60, 2, 18, -4), (24, 3, 15, -4), (80, 2, 1002, 26 - 35)]


@pytest.mark.parametrize("mode", [2, 3, 4])
@pytest.mark.parametrize("case", BLOCK_CASES)
def test_tma_register_blocks(qt, case, mode):
    """Every register-block shape of the tensor-copy GEMM (2 x 2, 2 x 4, 4 x 2, forced by
    QT_OPT_TMA = 2, 3, 4 wherever the tile allows it) against the FP64 oracle."""
    n, p, seed, off = case
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    net = qt.Network(edges, n, p, gammas, betas, z)
    qt.qt_set_option(net.handle, qt.QT_OPT_GEMM, 1)
    qt.qt_set_option(net.handle, qt.QT_OPT_TMA, mode)
    w = net.order(0)
    net.slice(w + off, 6, 1)
    net.prepare(0, batch=4)
    amp = net.contract(0)
    assert net.stats()["tma_gemm_launches"] > 0
    ref, _ = oracle_amplitude(tensors, norm, oracle_plan(adj, 0, w + off, 6, 1))
    assert rel_err(amp, ref) <= 1e-5, (mode, amp, ref)
