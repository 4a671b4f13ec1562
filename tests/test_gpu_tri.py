"""Triangle-form launches (three large tensors, every summed index in exactly two of
them) against the FP64 oracle, at the complex64 bar (rel.err <= 1e-5)."""

import pytest

from helpers import oracle_amplitude, oracle_plan, oracle_problem, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# n, p, seed, width offset (0: no slicing), batch; each plan has a triangle-form launch
CASES = [(36, 2, 7, 0, 1), (30, 3, 7, -2, 2), (50, 2, 2, -4, 3), (56, 2, 4, -2, 2),
         (44, 3, 1, -2, 1)]


def _run(qt, n, p, seed, off, batch, force):
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    net = qt.Network(edges, n, p, gammas, betas, z)
    qt.qt_set_option(net.handle, qt.QT_OPT_TRIANGLE, int(force))
    w = net.order(0)
    if off:
        net.slice(w + off, 6, 1)
        plan = oracle_plan(adj, 0, w + off, 6, 1)
    else:
        plan = oracle_plan(adj, 0)
    net.prepare(0, batch=batch)
    st = net.stats()
    net.upload()
    qt.qt_profile(net.handle, 1)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    net.run(0, 1 << len(plan["sliced"]), out)
    torch.cuda.synchronize()
    kinds = {r["kernel"] for r in qt.qt_profile_read(net.handle)}
    qt.qt_profile(net.handle, 0)
    amp = complex(out[0].item(), out[1].item())
    return amp, plan, tensors, norm, st, kinds


@pytest.mark.parametrize("case", CASES)
def test_triangle_form_matches_oracle(qt, case):
    amp, plan, tensors, norm, st, kinds = _run(qt, *case, force=True)
    assert st["tri_groups"] >= 1 and 6 in kinds
    ref, _ = oracle_amplitude(tensors, norm, plan)
    assert rel_err(amp, ref) <= 1e-5, (amp, ref, rel_err(amp, ref))
    amp0, *_ = _run(qt, *case, force=False)
    assert rel_err(amp0, ref) <= 1e-5


def test_triangle_form_bench_workload(qt):
    """N=80, p=2, seed 1002 sliced to width 26: its largest launch (a fused group of six
    buckets over three large tensors) in triangle form."""
    amp, plan, tensors, norm, st, kinds = _run(qt, 80, 2, 1002, 26 - 35, 4, force=True)
    assert 6 in kinds
    ref, _ = oracle_amplitude(tensors, norm, plan)
    assert rel_err(amp, ref) <= 1e-5, (amp, ref, rel_err(amp, ref))
