"""qt_contract_static: the contraction for callers that cannot allocate device memory.

Such a caller (a plugin inside an application that owns the CUDA allocator, or a
path that must not allocate) passes only inputs and outputs; the library keeps its
device scratch in one static array. These tests call the entry point through the C
ABI twice in a row and check each result against the workspace-based qt_contract on
the same network, within the tolerances of the other parity tests: with the default
kernels, and with the tensor-copy (TMA) GEMM and triangle kernels forced, whose
tensor maps then describe the static array. They also check that the caller's own
prepared schedule, upload and autotuned choices survive the static calls. The file
is named to run last.
"""

import pytest

from helpers import oracle_problem, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 4: 1e-10}


def _static_twice(qt, net, prec):
    stream = torch.cuda.current_stream().cuda_stream
    first = qt.qt_contract_static(net.handle, prec, stream)
    second = qt.qt_contract_static(net.handle, prec, stream)
    return first, second


@pytest.mark.parametrize("prec", [0, 4])
def test_static_matches_workspace_contract(qt, prec):
    n, p, seed = 24, 3, 15
    edges, gammas, betas, z, *_ = oracle_problem(n, p, seed)
    net = qt.Network(edges, n, p, gammas, betas, z)
    w = net.order(0)
    k, _ = net.slice(w - 4, 6, 1)
    assert k >= 1
    net.prepare(prec, batch=2)
    ref = net.contract(prec)
    net.autotune()
    first, second = _static_twice(qt, net, prec)
    assert rel_err(first, ref) <= TOL[prec], (first, ref)
    assert rel_err(second, ref) <= TOL[prec], (second, ref)
    # the caller's schedule, its upload to the caller's workspace and the autotuned
    # choices are untouched: a device-resident run needs no new qt_upload
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    net.run(0, 1 << k, out)
    torch.cuda.synchronize()
    again = complex(out[0].item(), out[1].item())
    assert rel_err(again, ref) <= TOL[prec]
    assert net.stats()["batch"] == 2


@pytest.mark.parametrize("form", ["gemm", "triangle"])
def test_static_tensor_copy_kernels(qt, form):
    """The TMA-staged GEMM (forced GEMM form) and triangle kernels on the static array."""
    n, p, seed, off = (44, 2, 14, -4) if form == "gemm" else (32, 3, 25, 0)
    edges, gammas, betas, z, *_ = oracle_problem(n, p, seed)
    net = qt.Network(edges, n, p, gammas, betas, z)
    qt.qt_set_option(net.handle, qt.QT_OPT_GEMM if form == "gemm" else qt.QT_OPT_TRIANGLE, 1)
    qt.qt_set_option(net.handle, qt.QT_OPT_TMA, 1)
    w = net.order(0)
    if off:
        net.slice(w + off, 6, 1)
    net.prepare(0, batch=2)
    ref = net.contract(0)
    before = net.stats()["tma_gemm_launches"]
    first, second = _static_twice(qt, net, 0)
    assert net.stats()["tma_gemm_launches"] > before  # the static calls took the TMA kernels
    assert rel_err(first, ref) <= 1e-5, (first, ref)
    assert rel_err(second, ref) <= 1e-5, (second, ref)


def test_static_rejects_oversized_network(qt):
    n, p, seed = 80, 2, 1002
    edges, gammas, betas, z, *_ = oracle_problem(n, p, seed)
    h = qt.qt_build_network(edges, n, p, gammas, betas, z)
    try:
        qt.qt_order(h, 0)
        qt.qt_slice(h, 26, 20, 1)  # rank-25 intermediates: ~680 MB per slice, beyond 64 MiB
        stream = torch.cuda.current_stream().cuda_stream
        with pytest.raises(qt.QtError) as e:
            qt.qt_contract_static(h, 0, stream)
        assert e.value.status == qt.QT_ENOMEM
        assert "static workspace holds" in str(e.value)
    finally:
        qt.qt_free(h)
