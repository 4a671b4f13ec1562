"""qt_contract_static: the contraction for callers that cannot allocate device memory.

Such a caller (a plugin inside an application that owns the CUDA allocator, or a
path that must not allocate) passes only inputs and outputs; the library keeps its
device scratch in one static array. This test calls the entry point through the C
ABI twice in a row and checks each result against the workspace-based qt_contract
on the same network, within the tolerances of the other parity tests. It is in a
file of its own so that it runs last.
"""

import pytest

from helpers import oracle_problem, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 4: 1e-10}


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
    stream = torch.cuda.current_stream().cuda_stream
    first = qt.qt_contract_static(net.handle, prec, stream)
    second = qt.qt_contract_static(net.handle, prec, stream)
    assert rel_err(first, ref) <= TOL[prec], (first, ref)
    assert rel_err(second, ref) <= TOL[prec], (second, ref)
    # the workspace path still works after the static one re-planned the batch
    again = net.contract(prec)
    assert rel_err(again, ref) <= TOL[prec]


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
