"""Segment launches (runs of small bucket launches executed by one block, or one
thread-block cluster, per slice) against the FP64 oracle, and against the same schedule
run one launch per group; every cluster size gives the same bits."""

import pytest

from helpers import oracle_amplitude, oracle_plan, oracle_problem, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 4: 1e-10}
CASES = [(14, 2, 7, 0, -3, 4, 1, 16), (24, 3, 15, 0, -4, 6, 1, 4), (44, 2, 14, 1, -4, 6, 1, 3),
         (60, 2, 18, 0, -4, 6, 2, 8)]


def _run(qt, case, prec, segments, cluster=0):
    n, p, seed, algo, off, mv, r, batch = case
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    net = qt.Network(edges, n, p, gammas, betas, z)
    qt.qt_set_option(net.handle, qt.QT_OPT_SEGMENTS, int(segments))
    qt.qt_set_option(net.handle, qt.QT_OPT_SEG_CLUSTER, cluster)
    w = net.order(algo)
    net.slice(max(1, w + off), mv, r)
    plan = oracle_plan(adj, algo, max(1, w + off), mv, r)
    net.prepare(prec, batch=batch)
    net.upload()
    qt.qt_profile(net.handle, 1)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    net.run(0, 1 << len(plan["sliced"]), out)
    torch.cuda.synchronize()
    kinds = [rec["kernel"] for rec in qt.qt_profile_read(net.handle)]
    qt.qt_profile(net.handle, 0)
    amp = complex(out[0].item(), out[1].item())
    ref, _ = oracle_amplitude(tensors, norm, plan)
    return amp, ref, kinds


@pytest.mark.parametrize("prec", [0, 4])
@pytest.mark.parametrize("case", CASES)
def test_segments_match_oracle_and_separate_launches(qt, case, prec):
    amp, ref, kinds = _run(qt, case, prec, True)
    amp0, _, kinds0 = _run(qt, case, prec, False)
    assert 5 in kinds and 5 not in kinds0
    assert len(kinds) < len(kinds0)
    assert rel_err(amp, ref) <= TOL[prec], (amp, ref)
    assert rel_err(amp0, ref) <= TOL[prec]
    # same arithmetic per element: the two runs differ at most by rounding
    assert abs(amp - amp0) <= TOL[prec] * abs(ref)


@pytest.mark.parametrize("prec", [0, 4])
@pytest.mark.parametrize("case", CASES)
def test_segment_cluster_sizes_same_bits(qt, case, prec):
    """Blocks per slice 1, 2, 4, 8: each result element is computed by one thread with
    the same arithmetic and the max-abs reductions are order-free, so the amplitude
    is bit-identical; also within tolerance of the oracle."""
    amps = {}
    for c in (1, 2, 4, 8):
        amp, ref, kinds = _run(qt, case, prec, True, cluster=c)
        assert 5 in kinds
        amps[c] = amp
    assert len(set(amps.values())) == 1, amps
    assert rel_err(amps[1], ref) <= TOL[prec], (amps[1], ref)


def test_segment_cluster_bench_shape(qt):
    """N=80, p=2, seed 1002 sliced to width 26 (4 slices in one batch): the automatic
    cluster size (8 blocks per slice) against one block per slice, bit for bit, and
    the oracle. Autotuning is left out so that both runs take the same kernels."""
    n, p, seed, algo, mv, r = 80, 2, 1002, 0, 20, 1
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    plan = oracle_plan(adj, algo, 26, mv, r)
    ref, _ = oracle_amplitude(tensors, norm, plan)
    amps = []
    for c in (0, 1):
        net = qt.Network(edges, n, p, gammas, betas, z)
        qt.qt_set_option(net.handle, qt.QT_OPT_SEG_CLUSTER, c)
        net.order(algo)
        k, _ = net.slice(26, mv, r)
        net.prepare(0, batch=1 << k)
        net.upload()
        out = torch.zeros(2, dtype=torch.float64, device="cuda")
        net.run(0, 1 << k, out)
        torch.cuda.synchronize()
        amps.append(complex(out[0].item(), out[1].item()))
    assert amps[0] == amps[1]
    assert rel_err(amps[0], ref) <= TOL[0]
