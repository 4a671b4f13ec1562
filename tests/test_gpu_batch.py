"""GPU parity for a batch of 2^a amplitudes with a open qubits (Sec. VII), through the
C ABI, against the FP64 oracle's open contraction.

Tolerance: the batch's norm-wise relative error max_b |x_b - r_b| / max_b |r_b| is at most
1e-5 for complex64 steps and 1e-10 for FP64 steps (the per-amplitude bounds of the
single-amplitude tests, applied to the batch as a vector).
"""

import numpy as np
import pytest

from helpers import batch_vector, oracle_amplitude, oracle_plan, oracle_problem_open

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 4: 1e-10}


def setup(qt, n, p, seed, opens, algo=0, drop=None, mv=0, r=1):
    (edges, gammas, betas, z, tensors, nv, norm, adj, keep,
     open_vars) = oracle_problem_open(n, p, seed, opens)
    net = qt.Network(edges, n, p, gammas, betas, z)
    net.set_open(opens)
    w = net.order(algo)
    lim, mvv = 1 << 30, 0
    if drop is not None:
        lim, mvv = max(1, w - drop), mv
        net.slice(lim, mvv, r)
    plan = oracle_plan(adj, algo, lim, mvv, r, keep)
    return net, plan, tensors, norm, open_vars


def normwise(x, ref):
    return np.max(np.abs(np.asarray(x) - ref)) / np.max(np.abs(ref))


CASES = [
    # n, p, seed, opens, algo, width drop (None: no slicing), max_vars, r, batch
    (10, 2, 2, [0], 0, None, 0, 1, 1),
    (12, 2, 3, [1, 5, 9], 1, 2, 4, 1, 3),
    (16, 3, 5, [0, 3, 6, 9, 12], 0, 3, 5, 1, 4),
    (24, 3, 15, [2, 4, 8, 16], 0, 4, 6, 1, 5),     # prefix and per-slice tiled launches
    (44, 2, 14, list(range(0, 44, 5)), 0, 4, 6, 1, 7),  # 9 open qubits, ragged batch
    (60, 2, 18, [7, 30, 59], 0, 4, 6, 2, 8),
]


@pytest.mark.parametrize("prec", [0, 4])
@pytest.mark.parametrize("case", CASES)
def test_batch_amplitudes(qt, case, prec):
    n, p, seed, opens, algo, drop, mv, r, batch = case
    net, plan, tensors, norm, ov = setup(qt, n, p, seed, opens, algo, drop, mv, r)
    net.prepare(prec, batch=batch)
    got = net.contract_batch(prec)
    assert len(got) == 1 << len(opens)
    ref, _ = oracle_amplitude(tensors, norm, plan, open_vars=ov)
    ref = batch_vector(ref, len(opens))
    assert normwise(got, ref) <= TOL[prec], normwise(got, ref)


@pytest.mark.parametrize("prec", [0, 4])
def test_batch_device_run_slice_ranges(qt, prec):
    """Device-resident runs over parts of the slice range add up to the oracle's per-slice
    tensors over those slices; two calls in a row give the same bits."""
    n, p, seed, opens = 24, 3, 15, [1, 11, 20]
    net, plan, tensors, norm, ov = setup(qt, n, p, seed, opens, 0, 4, 6, 1)
    k = len(plan["sliced"])
    assert k >= 2
    net.prepare(prec, batch=3)
    net.upload()
    a = len(opens)
    _, per = oracle_amplitude(tensors, norm, plan, open_vars=ov)
    out = torch.zeros(2 << a, dtype=torch.float64, device="cuda")
    for first, count in ((0, 1 << k), (1, (1 << k) - 2), (2, 1)):
        net.run(first, count, out)
        torch.cuda.synchronize()
        x = out.cpu().numpy()
        got = x[0::2] + 1j * x[1::2]
        ref = batch_vector(sum(per[first:first + count]), a)
        assert normwise(got, ref) <= TOL[prec]
        net.run(first, count, out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), x)


def test_batch_entry_matches_single_amplitude_network(qt):
    """Entry b of the batch equals the single-amplitude contraction of the bitstring with
    the open qubits set to b (both on the GPU, FP64)."""
    n, p, seed, opens = 20, 2, 9, [3, 12]
    net, plan, tensors, norm, ov = setup(qt, n, p, seed, opens)
    net.prepare(4, batch=1)
    got = net.contract_batch(4)
    from paper_2012_02430_gb300.inputs import qaoa_instance
    edges, gammas, betas, z = qaoa_instance(n, p, seed)
    for b in range(1 << len(opens)):
        zz = list(z)
        for j, v in enumerate(opens):
            zz[v] = (b >> j) & 1
        single = qt.Network(edges, n, p, gammas, betas, zz)
        single.order(0)
        single.prepare(4, batch=1)
        amp = single.contract(4)
        assert abs(amp - got[b]) <= 1e-10 * abs(amp)
