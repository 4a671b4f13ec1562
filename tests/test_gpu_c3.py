"""The mixed-precision configuration (p=3 QAOA on 3-regular graphs, Sec. VIII shapes)
against the FP64 oracle.

* N=120, p=3, seed 1003, sliced with 62 variables (64-bit slice ids; every slice fixes
  all of them after the first round's step, so a slice's widest step has 15 indices):
  seeded slice ids spread over [0, 2^62), each slice's value from qt_run(id, 1) against
  the oracle's value of the same slice, in FP32 and FP64. Slices are independent units
  of the amplitude (Eq. 2), so sampled slices measure the schedule at any size.
* N=50, p=3, seed 1003 stand-in: seeded bitstrings in every precision mode against the
  oracle's amplitude (split TF32 within the complex64 bar; plain TF32 and BF16 carry
  their input rounding of 10 and 8 mantissa bits).
"""

import pytest

from helpers import oracle_amplitude, oracle_plan, oracle_problem, rel_err
from oracle import contract, network
from paper_2012_02430_gb300.inputs import random_bitstring, random_slice_ids

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c3_net(qt):
    n, p, seed = 120, 3, 1003
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    net = qt.Network(edges, n, p, gammas, betas, z)
    net.order(0)
    k, _ = net.slice(28, 62, 1)
    assert k == 62
    sliced, step = qt.qt_get_slices(net.handle)
    order = qt.qt_get_order(net.handle)
    return net, tensors, norm, order, sliced, step


@pytest.mark.parametrize("prec", [0, 4])
def test_sampled_slices_n120_p3(qt, c3_net, prec):
    net, tensors, norm, order, sliced, step = c3_net
    ids = random_slice_ids(62, 3, 7) + [0, (1 << 62) - 1]
    net.prepare(prec, batch=1)
    net.upload()
    tol = 1e-5 if prec == 0 else 1e-10
    for sid in ids:
        out = torch.zeros(2, dtype=torch.float64, device="cuda")
        net.run(sid, 1, out)
        torch.cuda.synchronize()
        got = complex(out[0].item(), out[1].item())
        ref, _ = contract.contract_amplitude(tensors, order, sliced, step, [sid])
        ref *= norm
        assert rel_err(got, ref) <= tol, (prec, sid, got, ref)


TOL = {0: 1e-5, 3: 1e-5, 1: 1e-2, 2: 5e-2}
STAND_IN = (50, 3, 1003)
BITSTRINGS = [9000, 9001]


@pytest.fixture(scope="module")
def stand_in_refs():
    """The oracle's amplitude of each seeded bitstring (about 20 s each)."""
    n, p, seed = STAND_IN
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    from helpers import ALGO
    from oracle import ordering
    order, widths = ordering.greedy_order(adj, None, ALGO[0])
    w = max(widths)
    plan = oracle_plan(adj, 0, w - 6, 10, 1)
    refs = []
    for s in BITSTRINGS:
        zq = random_bitstring(n, s)
        t_q, _, norm_q = network.build_network(n, edges, p, gammas, betas, zq)
        refs.append((zq, oracle_amplitude(t_q, norm_q, plan)[0]))
    return edges, gammas, betas, w, refs


@pytest.mark.parametrize("prec", [0, 3, 1, 2])
def test_stand_in_n50_p3_bitstrings(qt, stand_in_refs, prec):
    n, p, seed = STAND_IN
    edges, gammas, betas, w, refs = stand_in_refs
    net = qt.Network(edges, n, p, gammas, betas, refs[0][0])
    assert net.order(0) == w
    net.slice(w - 6, 10, 1)
    net.prepare(prec, batch=4)
    for q, (zq, ref) in enumerate(refs):
        qt.qt_set_bitstring(net.handle, zq)
        amp = net.contract(prec)
        assert rel_err(amp, ref) <= TOL[prec], (prec, q, amp, ref, rel_err(amp, ref))
