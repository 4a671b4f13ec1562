"""GPU parity of launch paths the other files do not pin against the FP64 oracle:

* the benchmark workload exactly as the benchmark times it: autotuned kernel choice per
  launch, replayed from the captured CUDA graph with independent launches on four
  streams, in FP32 and in split-TF32 mode;
* the tiled kernel's scaled path (every operand times its exact power-of-two scale),
  forced in every slice (QT_OPT_SCALED), which natural QAOA magnitudes never reach;
* a contraction along a randomised greedy (rgreedy) order.
"""

import pytest

from helpers import oracle_amplitude, oracle_plan, oracle_problem, rel_err
from oracle import contract, rgreedy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run(qt, net, nslices):
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    net.run(0, nslices, out)
    torch.cuda.synchronize()
    return complex(out[0].item(), out[1].item())


@pytest.fixture(scope="module")
def bench_ref():
    n, p, seed = 80, 2, 1002
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    plan = oracle_plan(adj, 0, 26, 20, 1)
    ref, _ = oracle_amplitude(tensors, norm, plan)
    return (edges, gammas, betas, z), ref


@pytest.mark.parametrize("prec", [0, 3])
def test_bench_workload_as_timed(qt, bench_ref, prec):
    (edges, gammas, betas, z), ref = bench_ref
    net = qt.Network(edges, 80, 2, gammas, betas, z)
    net.order(0)
    k, _ = net.slice(26, 20, 1)
    net.prepare(prec, batch=1 << k)
    net.upload()
    tuned = net.autotune()
    assert len(tuned) > 0
    plan = qt.qt_launch_plan(net.handle)
    assert len({L["stream"] for L in plan["launches"]}) > 1  # the graph forks streams
    first = _run(qt, net, 1 << k)   # captures the graph
    second = _run(qt, net, 1 << k)  # replays it
    assert first == second
    assert rel_err(first, ref) <= 1e-5, (prec, first, ref, rel_err(first, ref))


def test_scaled_path_forced(qt, bench_ref):
    """Every tiled launch multiplies its operands by 2^-s_j: same amplitude within the
    complex64 bar, and the tiled kernel really ran."""
    (edges, gammas, betas, z), ref = bench_ref
    amps = {}
    for forced in (0, 1):
        net = qt.Network(edges, 80, 2, gammas, betas, z)
        qt.qt_set_option(net.handle, qt.QT_OPT_SCALED, forced)
        qt.qt_set_option(net.handle, qt.QT_OPT_SEGMENTS, 0)  # small steps on the tiled kernel too
        net.order(0)
        k, _ = net.slice(26, 20, 1)
        net.prepare(0, batch=1 << k)
        net.upload()
        qt.qt_profile(net.handle, 1)
        amps[forced] = _run(qt, net, 1 << k)
        kinds = {r["kernel"] for r in qt.qt_profile_read(net.handle)}
        qt.qt_profile(net.handle, 0)
        assert 1 in kinds
    assert rel_err(amps[1], ref) <= 1e-5, (amps[1], ref)
    assert rel_err(amps[1], amps[0]) <= 1e-5


@pytest.mark.parametrize("case", [(20, 2, 3, 0.2, 16), (30, 2, 9, 0.1, 32)])
def test_rgreedy_order_contraction(qt, case):
    """qt_order_rgreedy (bit-exact with the oracle's order on the CPU) then a GPU contraction
    along it: the amplitude of the oracle along the same order."""
    n, p, seed, tau, q = case
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    net = qt.Network(edges, n, p, gammas, betas, z)
    qt.qt_order_rgreedy(net.handle, tau, q, 17)
    order = qt.qt_get_order(net.handle)
    ro, _, _ = rgreedy.rgreedy_order(adj, tau, q, 17)
    assert list(order) == list(ro)
    net.prepare(0, batch=1)
    amp = net.contract(0)
    ref, _ = contract.contract_amplitude(tensors, ro)
    assert rel_err(amp, ref * norm) <= 1e-5, (amp, ref * norm)
