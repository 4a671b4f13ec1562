"""GPU parity: amplitudes from the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (stated by the method's accuracy targets): relative error <= 1e-5 for
complex64 steps, <= 1e-10 for FP64 steps; the relative error is
|a_gpu - a_ref| / |a_ref|.
"""

import pytest

from helpers import oracle_amplitude, oracle_plan, oracle_problem, rel_err
from oracle import statevector

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 4: 1e-10}


def gpu_network(qt, n, p, seed, algo=0, width_limit=None, max_vars=0, r=1):
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    net = qt.Network(edges, n, p, gammas, betas, z)
    w = net.order(algo)
    if width_limit is not None and max_vars > 0:
        net.slice(width_limit, max_vars, r)
    plan = oracle_plan(adj, algo, width_limit if width_limit is not None else 1 << 30,
                       max_vars if width_limit is not None else 0, r)
    return net, plan, tensors, norm, w


def run_device(qt, net, first, count):
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    net.run(first, count, out)
    torch.cuda.synchronize()
    return complex(out[0].item(), out[1].item())


@pytest.mark.parametrize("prec", [0, 4])
def test_c1_statevector(qt, prec):
    """N=20, p=1, no slicing: GPU vs the 2^20 statevector and the bucket oracle."""
    n, p, seed = 20, 1, 1001
    net, plan, tensors, norm, w = gpu_network(qt, n, p, seed)
    net.prepare(prec, batch=1)
    amp = net.contract(prec)
    edges, gammas, betas, z, *_ = oracle_problem(n, p, seed)
    sv = statevector.amplitude(n, edges, gammas, betas, z)
    ref, _ = oracle_amplitude(tensors, norm, plan)
    assert rel_err(ref, sv) < 1e-12
    assert rel_err(amp, sv) <= TOL[prec]


CASES = [
    # n, p, seed, algo, width_limit offset, max_vars, r, batch
    (8, 1, 1, 0, -2, 4, 1, 1),
    (10, 2, 2, 1, -2, 4, 1, 3),
    (12, 3, 3, 0, -3, 4, 2, 2),
    (14, 2, 7, 0, -3, 4, 1, 16),
    (16, 3, 5, 1, -4, 6, 1, 5),
    (24, 3, 15, 0, -4, 6, 1, 4),   # prefix steps reach the tiled kernel
    (44, 2, 14, 0, -4, 6, 1, 3),   # tiled kernel in the per-slice region, ragged batch
    (60, 2, 18, 0, -4, 6, 2, 8),
]


@pytest.mark.parametrize("prec", [0, 4])
@pytest.mark.parametrize("case", CASES)
def test_sliced_amplitude(qt, case, prec):
    n, p, seed, algo, off, mv, r, batch = case
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    net = qt.Network(edges, n, p, gammas, betas, z)
    w = net.order(algo)
    k, w2 = net.slice(max(1, w + off), mv, r)
    plan = oracle_plan(adj, algo, max(1, w + off), mv, r)
    assert len(plan["sliced"]) == k and plan["width"] == w2
    net.prepare(prec, batch=batch)
    amp = net.contract(prec)
    ref, _ = oracle_amplitude(tensors, norm, plan)
    assert rel_err(amp, ref) <= TOL[prec], (amp, ref)


@pytest.mark.parametrize("prec", [0, 4])
def test_slice_ranges_and_per_slice(qt, prec):
    """qt_run over sub-ranges: each slice against the oracle's per-slice value, and the
    sum of the ranges equals the full run (Eq. 2 on the device)."""
    n, p, seed = 16, 3, 5
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    net = qt.Network(edges, n, p, gammas, betas, z)
    w = net.order(0)
    k, _ = net.slice(w - 4, 3, 1)
    plan = oracle_plan(adj, 0, w - 4, 3, 1)
    assert k >= 2
    net.prepare(prec, batch=2)
    net.upload()
    total, per = oracle_amplitude(tensors, norm, plan)
    parts = []
    for sid in range(1 << k):
        a = run_device(qt, net, sid, 1)
        assert abs(a - per[sid]) <= TOL[prec] * abs(total) * 4, (sid, a, per[sid])
        parts.append(a)
    full = run_device(qt, net, 0, 1 << k)
    assert rel_err(full, total) <= TOL[prec]
    assert rel_err(sum(parts), full) <= TOL[prec]


def test_slice_sum_equals_unsliced_gpu(qt):
    """Eq. 2 on the GPU: the FP64 sliced sum equals the FP64 unsliced contraction."""
    n, p, seed = 44, 2, 14
    edges, gammas, betas, z, *_ = oracle_problem(n, p, seed)
    a = qt.Network(edges, n, p, gammas, betas, z)
    w = a.order(0)
    a.prepare(4, batch=1)
    unsliced = a.contract(4)
    b = qt.Network(edges, n, p, gammas, betas, z)
    b.order(0)
    k, _ = b.slice(w - 5, 6, 1)
    assert k >= 1
    b.prepare(4, batch=3)
    sliced = b.contract(4)
    assert rel_err(sliced, unsliced) <= 1e-10


@pytest.mark.parametrize("prec", [0, 4])
@pytest.mark.parametrize("case", [(24, 3, 15, -4), (44, 2, 14, -4), (60, 2, 18, -4)])
def test_fused_and_unfused_launches(qt, case, prec):
    """Fused launch groups (several indices summed per launch) and one launch per
    bucket give the oracle's amplitude."""
    n, p, seed, off = case
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    plan = None
    amps = {}
    for fuse in (0, 1):
        net = qt.Network(edges, n, p, gammas, betas, z)
        qt.qt_set_option(net.handle, qt.QT_OPT_FUSION, fuse)
        w = net.order(0)
        net.slice(w + off, 6, 1)
        if plan is None:
            plan = oracle_plan(adj, 0, w + off, 6, 1)
        net.prepare(prec, batch=3)
        st = net.stats()
        assert st["fused"] == fuse
        amps[fuse] = net.contract(prec)
    ref, _ = oracle_amplitude(tensors, norm, plan)
    for fuse in (0, 1):
        assert rel_err(amps[fuse], ref) <= TOL[prec], (fuse, amps[fuse], ref)


@pytest.mark.parametrize("prec", [0, 4])
def test_autotuned_schedule_parity(qt, prec):
    """Every kernel variant the autotuner may pick gives the oracle's amplitude."""
    n, p, seed = 60, 2, 18
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    net = qt.Network(edges, n, p, gammas, betas, z)
    w = net.order(0)
    net.slice(w - 4, 6, 1)
    plan = oracle_plan(adj, 0, w - 4, 6, 1)
    net.prepare(prec, batch=4)
    net.upload()
    report = net.autotune()
    assert report and all(0 <= r["variant"] <= 8 and len(r["ms"]) == 9 for r in report)
    ref, _ = oracle_amplitude(tensors, norm, plan)
    amp = net.contract(prec)
    assert rel_err(amp, ref) <= TOL[prec]


def test_no_edges_and_single_qubit(qt):
    """Degenerate graphs: no cost gates (closed form), one qubit."""
    import math
    for n, p in [(1, 1), (5, 2)]:
        gam = [0.3 * (k + 1) for k in range(p)]
        bet = [0.2 * (k + 1) for k in range(p)]
        z = [v % 2 for v in range(n)]
        net = qt.Network([], n, p, gam, bet, z)
        net.order(0)
        net.prepare(4, batch=1)
        amp = net.contract(4)
        # independent qubits: product of <z_v| prod_k exp(-i beta_k X) |+> = exp(-i sum beta) / sqrt 2
        ref = (complex(math.cos(sum(bet)), -math.sin(sum(bet))) / math.sqrt(2)) ** n
        assert abs(amp - ref) <= 1e-12


def test_set_angles_reuses_plan(qt):
    """The order and slices depend only on structure: new angles, same plan."""
    from paper_2012_02430_gb300.inputs import random_angles
    n, p, seed = 14, 2, 7
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    net = qt.Network(edges, n, p, gammas, betas, z)
    w = net.order(0)
    net.slice(w - 3, 4, 1)
    net.prepare(0, batch=4)
    net.contract(0)
    g2, b2 = random_angles(p, 99)
    qt.qt_set_angles(net.handle, g2, b2)
    amp = net.contract(0)
    from oracle import network
    t2, _, norm2 = network.build_network(n, edges, p, g2, b2, z)
    plan = oracle_plan(adj, 0, w - 3, 4, 1)
    ref, _ = oracle_amplitude(t2, norm2, plan)
    assert rel_err(amp, ref) <= 1e-5


def test_bench_workload_full(qt):
    """The benchmark workload at full size (N=80, p=2, seed 1002, sliced to rank 26,
    greedy min-fill): every slice on the GPU in the launch configuration the benchmark
    times, against the oracle's full complex128 sliced sum."""
    n, p, seed = 80, 2, 1002
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    net = qt.Network(edges, n, p, gammas, betas, z)
    net.order(0)
    k, w2 = net.slice(26, 20, 1)
    plan = oracle_plan(adj, 0, 26, 20, 1)
    assert w2 <= 26 and k == len(plan["sliced"])
    ref, _ = oracle_amplitude(tensors, norm, plan)
    for prec, batch in [(0, 1 << k), (4, 1)]:
        net.prepare(prec, batch=batch)
        amp = net.contract(prec)
        assert rel_err(amp, ref) <= TOL[prec], (prec, amp, ref)


def test_run_requires_current_upload(qt):
    """qt_run reads only an upload of the current schedule and angles: after qt_prepare,
    after new angles, or on another workspace it returns QT_ESTATE until qt_upload."""
    from paper_2012_02430_gb300.inputs import random_angles
    n, p, seed = 14, 2, 7
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    net = qt.Network(edges, n, p, gammas, betas, z)
    w = net.order(0)
    k, _ = net.slice(w - 3, 4, 1)
    plan = oracle_plan(adj, 0, w - 3, 4, 1)
    ref, _ = oracle_amplitude(tensors, norm, plan)
    net.prepare(0, batch=2)
    with pytest.raises(qt.QtError) as e:
        run_device(qt, net, 0, 1 << k)
    assert e.value.status == qt.QT_ESTATE
    net.upload()
    assert rel_err(run_device(qt, net, 0, 1 << k), ref) <= 1e-5
    net.prepare(0, batch=1)  # a new layout: the old upload no longer matches it
    with pytest.raises(qt.QtError) as e:
        run_device(qt, net, 0, 1 << k)
    assert e.value.status == qt.QT_ESTATE
    net.upload()
    assert rel_err(run_device(qt, net, 0, 1 << k), ref) <= 1e-5
    g2, b2 = random_angles(p, 99)
    qt.qt_set_angles(net.handle, g2, b2)
    with pytest.raises(qt.QtError) as e:
        run_device(qt, net, 0, 1 << k)
    assert e.value.status == qt.QT_ESTATE
    net.upload()
    from oracle import network
    t2, _, norm2 = network.build_network(n, edges, p, g2, b2, z)
    ref2, _ = oracle_amplitude(t2, norm2, plan)
    assert rel_err(run_device(qt, net, 0, 1 << k), ref2) <= 1e-5
    other = torch.empty_like(net.workspace)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(qt.QtError) as e:
        qt.qt_run(net.handle, 0, 1 << k, other.data_ptr(), other.numel(),
                  torch.cuda.current_stream().cuda_stream, out.data_ptr())
    assert e.value.status == qt.QT_ESTATE
