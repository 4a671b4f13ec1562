"""GEMM-form launches (pack kernels + batched complex GEMM) against the FP64 oracle:
CUDA-core FP32 and split-TF32 (3xTF32) tensor-core products must meet the complex64
bar (rel.err <= 1e-5); plain TF32 and BF16 tensor-core products carry their own input
rounding (10 and 8 mantissa bits) and are held to 1e-2 and 5e-2."""

import pytest

from helpers import oracle_amplitude, oracle_plan, oracle_problem, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32gemm": 1e-5, 3: 1e-5, 1: 1e-2, 2: 5e-2}
CASES = [(44, 2, 14, -4), (60, 2, 18, -4), (24, 3, 15, -4)]


def _amp(qt, n, p, seed, off, prec, force_gemm=False, profile=False, batch=3):
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    net = qt.Network(edges, n, p, gammas, betas, z)
    if force_gemm:
        qt.qt_set_option(net.handle, qt.QT_OPT_GEMM, int(force_gemm))
    w = net.order(0)
    net.slice(w + off, 6, 1)
    plan = oracle_plan(adj, 0, w + off, 6, 1)
    net.prepare(prec, batch=batch)
    st = net.stats()
    kinds = set()
    if profile:
        net.upload()
        qt.qt_profile(net.handle, 1)
        out = torch.zeros(2, dtype=torch.float64, device="cuda")
        net.run(0, 1 << len(plan["sliced"]), out)
        kinds = {r["kernel"] for r in qt.qt_profile_read(net.handle)}
        qt.qt_profile(net.handle, 0)
    amp = net.contract(prec)
    st = net.stats()
    ref, _ = oracle_amplitude(tensors, norm, plan)
    return amp, ref, st, kinds


@pytest.mark.parametrize("case", CASES)
def test_gemm_form_fp32_cuda_cores(qt, case):
    """FP32 GEMM form: the shared-memory tiled kernel (kind 4) where every summed index is
    in both big operands, the pack + CUDA-core GEMM (kind 3) elsewhere."""
    amp, ref, st, kinds = _amp(qt, *case, 0, force_gemm=True, profile=True)
    assert st["gemm_groups"] >= 1 and kinds & {3, 4, 7}
    assert rel_err(amp, ref) <= TOL["fp32gemm"], (amp, ref)


def test_gemm_tile_bench_workload(qt):
    """N=80, p=2, seed 1002 sliced to width 26, every GEMM-form launch forced: the tiled
    GEMM kernel runs and the amplitude meets the complex64 bar."""
    amp, ref, st, kinds = _amp(qt, 80, 2, 1002, 26 - 35, 0, force_gemm=True, profile=True)
    assert 4 in kinds
    assert rel_err(amp, ref) <= TOL["fp32gemm"], (amp, ref)


STREAM_CASES = [(44, 2, 14, -4, 3), (60, 2, 18, -4, 3), (80, 2, 1002, 26 - 35, 4),
                (50, 3, 1003, -4, 2)]


@pytest.mark.parametrize("case", STREAM_CASES)
def test_gemm_stream_kernel(qt, case):
    """GEMM form with the streaming kernel forced where it applies (QT_OPT_GEMM = 2: the
    small operand staged whole per slice, one thread per row of the large one), the
    tiled GEMM elsewhere: the amplitude meets the complex64 bar and the streaming
    kernel really ran."""
    n, p, seed, off, batch = case
    amp, ref, st, kinds = _amp(qt, n, p, seed, off, 0, force_gemm=2, batch=batch)
    assert st["stream_gemm_launches"] > 0
    assert rel_err(amp, ref) <= TOL["fp32gemm"], (amp, ref)


@pytest.mark.parametrize("prec", [3, 1, 2])
@pytest.mark.parametrize("case", CASES)
def test_gemm_form_tensor_cores(qt, case, prec):
    """TF32 and split-TF32 modes: GEMM-form launches on the tcgen05 kernel where it
    applies (profile class 8), the FP32 GEMM elsewhere; BF16: the warp-level mma.sync
    kernel (pack + GEMM, class 3)."""
    amp, ref, st, kinds = _amp(qt, *case, prec, profile=True)
    assert st["gemm_groups"] >= 1 and kinds & ({3} if prec == 2 else {3, 4, 8})
    assert rel_err(amp, ref) <= TOL[prec], (prec, amp, ref, rel_err(amp, ref))


@pytest.mark.parametrize("prec", [3, 1])
@pytest.mark.parametrize("case", CASES)
def test_gemm_form_legacy_mma_sync(qt, case, prec):
    """QT_OPT_TCGEN05 = 2: TF32 modes on the warp-level mma.sync kernels."""
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(case[0], case[1], case[2])
    net = qt.Network(edges, case[0], case[1], gammas, betas, z)
    qt.qt_set_option(net.handle, qt.QT_OPT_TCGEN05, 2)
    w = net.order(0)
    net.slice(w + case[3], 6, 1)
    net.prepare(prec, batch=3)
    amp = net.contract(prec)
    assert net.stats()["tcgen05_gemm_launches"] == 0
    ref, _ = oracle_amplitude(tensors, norm, oracle_plan(adj, 0, w + case[3], 6, 1))
    assert rel_err(amp, ref) <= TOL[prec], (prec, rel_err(amp, ref))


@pytest.mark.parametrize("prec", [3, 1, 2])
def test_bench_workload_tensor_core_modes(qt, prec):
    """N=80, p=2, seed 1002 sliced to width 26: 69% of the ledger's flops sit in launches
    with full 16 x 8 tensor-core tiles."""
    amp, ref, st, _ = _amp(qt, 80, 2, 1002, 26 - 35, prec)
    assert st["tensor_core_shape_flops"] > 0.5 * st["job_flops"]
    assert rel_err(amp, ref) <= TOL[prec], (prec, rel_err(amp, ref))
