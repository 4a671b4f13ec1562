"""GEMM-form launches on the tcgen05 tensor cores against the FP64 oracle.

The kernel (operand rows loaded by TMA tensor copies, split-TF32 planes in shared
memory, products accumulated in tensor memory, outputs staged in shared memory and
written as contiguous runs) is forced on every launch it applies to
(QT_OPT_TCGEN05 = 1, and 3 for the other tile shape). The cases reach every way the
two lowest output indices can fall on group and column indices, summed-index counts
2 to 6, both choices of the side that gives the 128 tensor-memory lanes, and work units
that carry a chunk of the summed values (rows too long for shared memory, or forced
with QT_OPT_TCGEN05 = 4). Split
TF32 (3 products per input pair) must meet the complex64 bar, 1e-5; plain TF32 (one
product of 10-bit-mantissa inputs) is held to 1e-2.
"""

import pytest

from helpers import oracle_amplitude, oracle_plan, oracle_problem, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {3: 1e-5, 1: 1e-2}

# (n, p, seed, width offset) -> (how output bits 0 and 1 fall, summed indices, lane side)
CASES = [
    (30, 3, 5, -4),    # (0, 2, A)
    (44, 2, 3, -2),    # (0, 3, A)
    (60, 2, 19, -4),   # (0, 4, A) and (2, 4, A)
    (48, 2, 14, -2),   # (1, 2, A)
    (50, 2, 7, -2),    # (1, 2, B)
    (48, 2, 5, 0),     # (1, 3, A)
    (48, 2, 24, -4),   # (1, 4, A)
    (44, 3, 15, -2),   # (1, 5, A)
    (50, 2, 22, -4),   # (2, 2, A)
    (50, 2, 23, -2),   # (2, 3, A)
    (30, 3, 21, -2),   # (3, 2, A)
    (24, 3, 21, 0),    # (3, 3, A)
    (40, 3, 21, -4),   # (3, 4, A)
]


def _net(qt, n, p, seed, off, force=1):
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    net = qt.Network(edges, n, p, gammas, betas, z)
    qt.qt_set_option(net.handle, qt.QT_OPT_TCGEN05, force)
    w = net.order(0)
    if off:
        net.slice(w + off, 6, 1)
    plan = oracle_plan(adj, 0, w + off, 6, 1) if off else oracle_plan(adj, 0)
    return net, tensors, norm, plan


def _umma_launches(qt, net):
    lp = qt.qt_launch_plan(net.handle)
    return [L["umma"] for L in lp["launches"] if "umma" in L]


@pytest.mark.parametrize("force", [1, 3])
@pytest.mark.parametrize("case", CASES)
def test_umma_split_tf32_matches_oracle(qt, case, force):
    """Both tile shapes: the widest products (1) and the longest output runs (3)."""
    net, tensors, norm, plan = _net(qt, *case, force=force)
    net.prepare(3, batch=2)
    plans = _umma_launches(qt, net)
    assert plans, "no launch takes the tcgen05 kernel"
    amp = net.contract(3)  # QT_ETIMEOUT if a bounded wait gave up
    assert net.stats()["tcgen05_gemm_launches"] > 0
    ref, _ = oracle_amplitude(tensors, norm, plan)
    assert rel_err(amp, ref) <= TOL[3], (case, amp, ref, rel_err(amp, ref))


# rows too long for shared memory: the summed values in chunks accumulated in tensor memory
CHUNK_CASES = [(36, 3, 14, 0),   # 6 summed indices (K = 64), chunks of 16
               (30, 3, 7, 0)]    # 5 summed indices, chunks of 8


@pytest.mark.parametrize("case", CHUNK_CASES)
def test_umma_chunked_summed_values(qt, case):
    """Launches whose whole rows do not fit: the plan takes chunks of the summed values
    (kc < nsum), and the split-TF32 amplitude meets the complex64 bar."""
    net, tensors, norm, plan = _net(qt, *case)
    net.prepare(3, batch=2)
    plans = _umma_launches(qt, net)
    assert any(u["kc"] < u["nsum"] for u in plans), plans
    amp = net.contract(3)
    assert net.stats()["tcgen05_gemm_launches"] > 0
    ref, _ = oracle_amplitude(tensors, norm, plan)
    assert rel_err(amp, ref) <= TOL[3], (case, amp, ref, rel_err(amp, ref))


@pytest.mark.parametrize("case", CASES[:6] + CHUNK_CASES)
def test_umma_forced_small_chunks(qt, case):
    """QT_OPT_TCGEN05 = 4: every work unit carries 4 summed values, so every launch
    accumulates its products over several chunks; split TF32 within 1e-5."""
    net, tensors, norm, plan = _net(qt, *case, force=4)
    net.prepare(3, batch=2)
    plans = _umma_launches(qt, net)
    assert plans and all(u["kc"] == 2 for u in plans), plans
    amp = net.contract(3)
    assert net.stats()["tcgen05_gemm_launches"] > 0
    ref, _ = oracle_amplitude(tensors, norm, plan)
    assert rel_err(amp, ref) <= TOL[3], (case, amp, ref, rel_err(amp, ref))


@pytest.mark.parametrize("case", CASES[:4])
def test_umma_plain_tf32(qt, case):
    net, tensors, norm, plan = _net(qt, *case)
    net.prepare(1, batch=2)
    amp = net.contract(1)
    assert net.stats()["tcgen05_gemm_launches"] > 0
    ref, _ = oracle_amplitude(tensors, norm, plan)
    assert rel_err(amp, ref) <= TOL[1], (case, rel_err(amp, ref))


def test_umma_repeatable_and_slice_ranges(qt):
    """Two runs give the same bits; per-slice runs (qt_run sub-ranges) sum to the whole."""
    net, tensors, norm, plan = _net(qt, 60, 2, 19, -4)
    k = len(plan["sliced"])
    net.prepare(3, batch=1 << k)
    net.upload()
    outs = []
    for first, count in [(0, 1 << k), (0, 1 << k)] + [(s, 1) for s in range(1 << k)]:
        out = torch.zeros(2, dtype=torch.float64, device="cuda")
        net.run(first, count, out)
        torch.cuda.synchronize()
        outs.append(complex(out[0].item(), out[1].item()))
    assert outs[0] == outs[1]
    ref, per = oracle_amplitude(tensors, norm, plan)
    for s in range(1 << k):
        assert rel_err(outs[2 + s], per[s]) <= TOL[3], (s, outs[2 + s], per[s])
    assert rel_err(sum(outs[2:]), ref) <= TOL[3]


def test_umma_bench_workload(qt):
    """N=80, p=2, seed 1002 sliced to width 26 (all 4 slices in one batch): the tcgen05
    kernel forced on every GEMM-form launch it takes, then the same after the
    autotuner chose per launch among it and the FP32 kernels; both within 1e-5."""
    n, p, seed = 80, 2, 1002
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    plan = oracle_plan(adj, 0, 26, 20, 1)
    ref, _ = oracle_amplitude(tensors, norm, plan)
    for force in (1, 0):
        net = qt.Network(edges, n, p, gammas, betas, z)
        qt.qt_set_option(net.handle, qt.QT_OPT_TCGEN05, force)
        net.order(0)
        k, w2 = net.slice(26, 20, 1)
        net.prepare(3, batch=1 << k)
        assert len(_umma_launches(qt, net)) >= 2
        net.upload()
        if force == 0:
            net.autotune()
        out = torch.zeros(2, dtype=torch.float64, device="cuda")
        net.run(0, 1 << k, out)
        torch.cuda.synchronize()
        amp = complex(out[0].item(), out[1].item())
        assert rel_err(amp, ref) <= TOL[3], (force, amp, ref, rel_err(amp, ref))
        if force == 1:
            assert net.stats()["tcgen05_gemm_launches"] >= 2
