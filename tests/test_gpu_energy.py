"""Batched lightcone energy on the GPU (one persistent launch) against the FP64 oracle:
per-edge <Z_u Z_v> from the oracle's lightcone contractions, the 2^N statevector energy
for small graphs and the closed-form p=1 edge energy (with its triangle term)."""

import itertools
import math

import pytest

from oracle import energy, statevector
from paper_2012_02430_gb300.inputs import qaoa_instance

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 4: 1e-10}  # on <Z_u Z_v> in [-1, 1] and on the energy relative to |E|


def gpu_energy(qt, n, edges, p, g, b, prec, algo=0, tune=False):
    en = qt.Energy(edges, n, p, g, b, algo)
    en.prepare(prec)
    if tune:
        en.upload()
        en.autotune()
    return en.compute(prec), en


@pytest.mark.parametrize("prec", [0, 4])
@pytest.mark.parametrize("n,p,seed", [(12, 1, 5), (14, 2, 6), (12, 3, 7)])
def test_energy_small_vs_statevector(qt, n, p, seed, prec):
    edges, g, b, z = qaoa_instance(n, p, seed)
    (E, zz), _ = gpu_energy(qt, n, edges, p, g, b, prec)
    e_sv = statevector.maxcut_energy(n, edges, g, b)
    zz_sv = statevector.zz_expectations(n, edges, g, b)
    assert abs(E - e_sv) <= TOL[prec] * abs(e_sv)
    assert max(abs(x - y) for x, y in zip(zz, zz_sv)) <= TOL[prec]


@pytest.mark.parametrize("prec", [0, 4])
def test_energy_p1_closed_form_with_triangles(qt, prec):
    n = 7
    edges = [(0, 1), (1, 2), (0, 2), (2, 3), (3, 4), (4, 5), (3, 5), (5, 6), (0, 6), (1, 4)]
    g, b = [0.77], [0.31]
    (E, zz), _ = gpu_energy(qt, n, edges, 1, g, b, prec)
    for (u, v), x in zip(edges, zz):
        cf = energy.edge_energy_p1_closed_form(n, edges, g[0], b[0], u, v)
        assert abs(0.5 * (1 - x) - cf) <= TOL[prec]


@pytest.mark.parametrize("prec", [0, 4])
def test_energy_batched_workload_full(qt, prec):
    """The batched-energy workload at full size: p=2 on a random 3-regular graph with
    N=1000 (seed 1004), 1500 lightcone networks in one persistent launch, every edge
    against the oracle; the autotuned launch shape must not change the result."""
    n, p, seed = 1000, 2, 1004
    edges, g, b, z = qaoa_instance(n, p, seed)
    E_ref, zz_ref = energy.energy_lightcone(n, edges, p, g, b)
    (E, zz), en = gpu_energy(qt, n, edges, p, g, b, prec, tune=True)
    assert max(abs(x - y) for x, y in zip(zz, zz_ref)) <= TOL[prec]
    assert abs(E - E_ref) <= TOL[prec] * abs(E_ref)
    st = en.stats()
    assert st["edges"] == 1500 and st["max_width"] >= 4


def test_energy_p1_closed_form_regular_full(qt):
    """p=1 variant of the batched workload: every edge against the closed form."""
    n, seed = 1000, 1004
    edges, g, b, z = qaoa_instance(n, 1, seed)
    (E, zz), _ = gpu_energy(qt, n, edges, 1, g, b, 0)
    cf = [energy.edge_energy_p1_closed_form(n, edges, g[0], b[0], u, v) for u, v in edges]
    assert max(abs(0.5 * (1 - x) - c) for x, c in zip(zz, cf)) <= 1e-5
    assert abs(E - sum(cf)) <= 1e-5 * sum(cf)


def test_energy_set_angles(qt):
    n, p, seed = 14, 2, 8
    edges, g, b, z = qaoa_instance(n, p, seed)
    en = qt.Energy(edges, n, p, g, b)
    en.prepare(0)
    en.compute(0)
    g2, b2 = [0.4, 1.1], [2.0, 0.7]
    qt.qt_energy_set_angles(en.handle, g2, b2)
    E, zz = en.compute(0)
    assert abs(E - statevector.maxcut_energy(n, edges, g2, b2)) <= 1e-5 * abs(E)


def test_energy_device_run(qt):
    n, p, seed = 30, 2, 12
    edges, g, b, z = qaoa_instance(n, p, seed)
    en = qt.Energy(edges, n, p, g, b)
    en.prepare(0)
    en.upload()
    zz = torch.zeros(len(edges), dtype=torch.float64, device="cuda")
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(3):
        en.run(zz, E)
    torch.cuda.synchronize()
    E_ref, zz_ref = energy.energy_lightcone(n, edges, p, g, b)
    assert abs(E.item() - E_ref) <= 1e-5 * abs(E_ref)
    assert max(abs(x - y) for x, y in zip(zz.tolist(), zz_ref)) <= 1e-5


@pytest.mark.parametrize("prec", [0, 4])
def test_energy_angle_sweep_vs_statevector(qt, prec):
    """Angle sweep: 6 angle sets of one N=14, p=2 graph in one persistent launch; each
    set's energy and <Z_u Z_v> equal the 2^14 statevector's."""
    from paper_2012_02430_gb300.inputs import random_angles
    n, p, seed = 14, 2, 6
    edges, g, b, z = qaoa_instance(n, p, seed)
    en = qt.Energy(edges, n, p, g, b)
    en.prepare(prec)
    sets = [random_angles(p, 300 + s) for s in range(6)]
    en.sweep_prepare(len(sets))
    E = torch.zeros(len(sets), dtype=torch.float64, device="cuda")
    zz = torch.zeros(len(sets), len(edges), dtype=torch.float64, device="cuda")
    en.sweep([s[0] for s in sets], [s[1] for s in sets], E, zz)
    torch.cuda.synchronize()
    for q, (gs, bs) in enumerate(sets):
        e_sv = statevector.maxcut_energy(n, edges, gs, bs)
        zz_sv = statevector.zz_expectations(n, edges, gs, bs)
        assert abs(E[q].item() - e_sv) <= TOL[prec] * abs(e_sv)
        assert max(abs(zz[q, i].item() - zz_sv[i]) for i in range(len(edges))) <= TOL[prec]


def test_energy_angle_sweep_matches_single_runs(qt):
    """N=200, p=2: a sweep of 4 angle sets gives each set's single-run energy and the
    oracle's lightcone energy."""
    from paper_2012_02430_gb300.inputs import random_angles
    n, p, seed = 200, 2, 1004
    edges, g, b, z = qaoa_instance(n, p, seed)
    en = qt.Energy(edges, n, p, g, b)
    en.prepare(0)
    sets = [random_angles(p, 400 + s) for s in range(4)]
    en.sweep_prepare(len(sets))
    E = torch.zeros(len(sets), dtype=torch.float64, device="cuda")
    en.sweep([s[0] for s in sets], [s[1] for s in sets], E)
    torch.cuda.synchronize()
    for q, (gs, bs) in enumerate(sets):
        E_ref, _ = energy.energy_lightcone(n, edges, p, gs, bs)
        assert abs(E[q].item() - E_ref) <= TOL[0] * abs(E_ref)
        single = qt.Energy(edges, n, p, gs, bs)
        single.prepare(0)
        e1, _ = single.compute(0)
        assert abs(E[q].item() - e1) <= 1e-9 * abs(e1)
