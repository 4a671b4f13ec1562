"""A plan made by the learned slicing search (the committed GPU-trained proposal model
verifies its top candidates per round; greedy ordering decides) contracted on the GPU:
the amplitude of the oracle along the same order and slices."""

import pytest

from helpers import oracle_problem, rel_err
from oracle import contract

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", [(30, 2, 5, -3, 4), (40, 2, 8, -4, 6)])
def test_learned_plan_contraction(qt, case):
    import ctypes as C

    import numpy as np

    from paper_2012_02430_gb300 import learn
    params, hidden, _ = learn.load()
    n, p, seed, drop, max_vars = case
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    net = qt.Network(edges, n, p, gammas, betas, z)
    w = net.order(0)
    pa = np.ascontiguousarray(params, dtype=np.float32)
    k, wd = C.c_int32(), C.c_int32()
    qt._check(qt.lib.qt_slice_learned(net.handle, pa.ctypes.data_as(C.POINTER(C.c_float)), hidden,
                                      w + drop, max_vars, 1, 3, 8, 0, C.byref(k), C.byref(wd)))
    assert k.value >= 1
    order = qt.qt_get_order(net.handle)
    sliced, step = qt.qt_get_slices(net.handle)
    net.prepare(0, batch=1 << k.value)
    amp = net.contract(0)
    ref, _ = contract.contract_amplitude(tensors, order, sliced, step)
    assert rel_err(amp, ref * norm) <= 1e-5, (amp, ref * norm)
