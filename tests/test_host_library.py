"""The C-ABI library on the CPU: exported symbols, bit-exact integer plans against the
oracle (network, orders, widths, slices, ledger), and argument/state error handling."""

import math
import re
import os

import pytest

from helpers import oracle_plan, oracle_problem, oracle_problem_open
from oracle import ledger

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    with open(os.path.join(ROOT, "include", "qtensor.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^(?:qt_status|void|const char\*)\s+(qt_\w+)\(", text, re.M)))


def test_library_exports_every_header_symbol(qt):
    names = header_symbols()
    assert len(names) >= 20
    for name in names:
        assert hasattr(qt.lib, name), name
    assert "sm_103a" in qt.qt_version()


def test_network_tensors_match_oracle(qt):
    n, p, seed = 10, 3, 4
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    h = qt.qt_build_network(edges, n, p, gammas, betas, z)
    try:
        cnt, nvars = qt.qt_num_tensors(h)
        assert cnt == len(tensors) and nvars == nv
        for t, (labels, data) in enumerate(tensors):
            lab, flat = qt.qt_get_tensor(h, t)
            assert tuple(lab) == tuple(labels)
            r = len(lab)
            for e in range(1 << r):
                idx = tuple((e >> a) & 1 for a in range(r))  # axis a = bit a of e
                want = data[idx]
                assert abs(complex(flat[2 * e], flat[2 * e + 1]) - want) < 1e-15
    finally:
        qt.qt_free(h)


CASES = [(8, 1, 1, 3, 4, 1), (12, 3, 3, 8, 4, 1), (12, 3, 3, 8, 4, 2), (20, 1, 1001, 3, 4, 1),
         (30, 2, 11, 12, 6, 1), (24, 3, 15, 14, 6, 2), (44, 2, 14, 17, 6, 1)]


@pytest.mark.parametrize("algo", [0, 1])
@pytest.mark.parametrize("case", CASES)
def test_plan_bit_exact(qt, case, algo):
    n, p, seed, lim, mv, r = case
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    h = qt.qt_build_network(edges, n, p, gammas, betas, z)
    try:
        from oracle import ordering
        o, w = ordering.greedy_order(adj, None, {0: ordering.MIN_FILL, 1: ordering.MIN_DEGREE}[algo])
        assert qt.qt_order(h, algo) == max(w)
        assert qt.qt_get_order(h) == o and qt.qt_get_widths(h) == w
        plan = oracle_plan(adj, algo, lim, mv, r)
        k, width = qt.qt_slice(h, lim, mv, r)
        sliced, step = qt.qt_get_slices(h)
        assert sliced == plan["sliced"] and step == plan["slice_step"]
        assert qt.qt_get_order(h) == plan["order"] and qt.qt_get_widths(h) == plan["widths"]
        assert width == plan["width"] and k == len(plan["sliced"])
        for prec, eb in ((0, 8), (4, 16)):
            qt.qt_prepare(h, prec, 3)
            st = qt.qt_stats(h)
            tot, steps = ledger.ledger([l for l, _ in tensors], plan["order"], plan["sliced"],
                                       plan["slice_step"])
            for key in ("prefix_flops", "prefix_bytes", "slice_flops", "slice_bytes",
                        "prefix_width", "slice_width", "n_prefix_steps", "n_slice_steps"):
                assert st[key] == tot[key], key
            assert [s[2:5] for s in st["steps"]] == [[s["m"], s["u"], s["c"]] for s in steps]
            groups = ledger.launch_groups([l for l, _ in tensors], plan["order"], plan["sliced"],
                                          plan["slice_step"])
            assert st["groups"] == groups
            assert sum(g[6] for g in groups) == tot["prefix_flops"] + tot["slice_flops"]
            assert st["nslices"] == 1 << k and st["batch"] == min(3, 1 << k)
            assert st["elem_bytes"] == eb
    finally:
        qt.qt_free(h)


@pytest.mark.slow
def test_bench_workload_plan_bit_exact(qt):
    """The benchmark workload's plan (N=80, p=2, seed 1002, width <= 26): order, slices, ledger."""
    n, p, seed = 80, 2, 1002
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    h = qt.qt_build_network(edges, n, p, gammas, betas, z)
    try:
        qt.qt_order(h, 0)
        k, width = qt.qt_slice(h, 26, 20, 1)
        plan = oracle_plan(adj, 0, 26, 20, 1)
        assert qt.qt_get_slices(h) == (plan["sliced"], plan["slice_step"])
        assert qt.qt_get_order(h) == plan["order"] and width == plan["width"] <= 26
        qt.qt_prepare(h, 0, 1 << k)
        st = qt.qt_stats(h)
        tot, _ = ledger.ledger([l for l, _ in tensors], plan["order"], plan["sliced"],
                               plan["slice_step"])
        assert st["slice_flops"] == tot["slice_flops"] and st["slice_bytes"] == tot["slice_bytes"]
        groups = ledger.launch_groups([l for l, _ in tensors], plan["order"], plan["sliced"],
                                      plan["slice_step"])
        assert st["groups"] == groups
    finally:
        qt.qt_free(h)


def test_errors(qt):
    QtError = qt.QtError
    g, b = [0.1], [0.2]
    with pytest.raises(QtError) as e:
        qt.qt_build_network([(0, 0)], 2, 1, g, b, [0, 0])
    assert e.value.status == qt.QT_EINVAL
    with pytest.raises(QtError) as e:
        qt.qt_build_network([(0, 1), (1, 0)], 2, 1, g, b, [0, 0])
    assert e.value.status == qt.QT_EINVAL
    with pytest.raises(QtError) as e:
        qt.qt_build_network([(0, 5)], 2, 1, g, b, [0, 0])
    assert e.value.status == qt.QT_EINVAL
    with pytest.raises(QtError) as e:
        qt.qt_build_network([(0, 1)], 2, 1, g, b, [0, 2])
    assert e.value.status == qt.QT_EINVAL
    with pytest.raises(QtError) as e:
        qt.qt_build_network([(0, 1)], 2, 1, [math.nan], b, [0, 1])
    assert e.value.status == qt.QT_EINVAL
    h = qt.qt_build_network([(0, 1), (1, 2)], 3, 1, g, b, [0, 1, 0])
    try:
        for call in (lambda: qt.qt_slice(h, 2, 1), lambda: qt.qt_prepare(h, 0, 1),
                     lambda: qt.qt_get_order(h), lambda: qt.qt_stats(h)):
            with pytest.raises(QtError) as e:
                call()
            assert e.value.status == qt.QT_ESTATE
        qt.qt_order(h, 0)
        with pytest.raises(QtError) as e:
            qt.qt_order(h, 7)
        assert e.value.status == qt.QT_EINVAL
        with pytest.raises(QtError) as e:
            qt.qt_slice(h, 0, 1)
        assert e.value.status == qt.QT_EINVAL
        with pytest.raises(QtError) as e:
            qt.qt_prepare(h, 7, 1)
        assert e.value.status == qt.QT_EINVAL
        need = qt.qt_prepare(h, 0, 1)
        assert need > 0
        # workspace checks happen before any CUDA call
        with pytest.raises(QtError) as e:
            qt.qt_run(h, 0, 1, 0, need, 0, 0)
        assert e.value.status == qt.QT_EINVAL
        with pytest.raises(QtError) as e:
            qt.qt_run(h, 0, 2, 256, need, 0, 256)
        assert e.value.status == qt.QT_EINVAL
        with pytest.raises(QtError) as e:
            qt.qt_run(h, 0, 1, 256 * 3 + 8, need, 0, 256)
        assert e.value.status == qt.QT_EINVAL
        with pytest.raises(QtError) as e:
            qt.qt_run(h, 0, 1, 256, need - 1, 0, 256)
        assert e.value.status == qt.QT_ENOMEM
        # a workspace that never received qt_upload for this schedule: refused before any
        # CUDA call, so a stale layout is never read
        with pytest.raises(QtError) as e:
            qt.qt_run(h, 0, 1, 256, need, 0, 256)
        assert e.value.status == qt.QT_ESTATE
        assert "qt_upload" in str(e.value)
        with pytest.raises(QtError) as e:
            qt.qt_autotune(h, 256, need, 0)
        assert e.value.status == qt.QT_ESTATE
    finally:
        qt.qt_free(h)


OPEN_CASES = [(8, 1, 1, [0], 3, 4, 1), (12, 2, 3, [5, 1], 7, 4, 1), (12, 3, 3, [2, 9, 4], 8, 4, 2),
              (24, 2, 15, [0, 23, 7, 11], 10, 6, 1), (30, 2, 11, [3, 4, 5, 6, 7, 8], 12, 6, 1)]


@pytest.mark.parametrize("algo", [0, 1])
@pytest.mark.parametrize("case", OPEN_CASES)
def test_open_plan_bit_exact(qt, case, algo):
    """Open qubits (Sec. VII): tensors, greedy order, slicing plan and launch groups of the
    library equal the oracle's, the open variables never eliminated nor sliced."""
    n, p, seed, opens, lim, mv, r = case
    (edges, gammas, betas, z, tensors, nv, norm, adj, keep,
     open_vars) = oracle_problem_open(n, p, seed, opens)
    h = qt.qt_build_network(edges, n, p, gammas, betas, z)
    try:
        qt.qt_set_open(h, opens)
        cnt, nvars = qt.qt_num_tensors(h)
        assert cnt == len(tensors) and nvars == nv
        for t, (labels, data) in enumerate(tensors):
            lab, flat = qt.qt_get_tensor(h, t)
            assert tuple(lab) == tuple(labels)
            for e in range(1 << len(lab)):
                want = data[tuple((e >> x) & 1 for x in range(len(lab)))]
                assert abs(complex(flat[2 * e], flat[2 * e + 1]) - want) < 1e-15
        from oracle import ordering
        o, w = ordering.greedy_order(adj, None, {0: ordering.MIN_FILL, 1: ordering.MIN_DEGREE}[algo],
                                     keep)
        assert qt.qt_order(h, algo) == max(w)
        assert qt.qt_get_order(h) == o and qt.qt_get_widths(h) == w
        plan = oracle_plan(adj, algo, lim, mv, r, keep)
        k, width = qt.qt_slice(h, lim, mv, r)
        assert qt.qt_get_slices(h) == (plan["sliced"], plan["slice_step"])
        assert qt.qt_get_order(h) == plan["order"] and width == plan["width"]
        assert not set(plan["order"] + plan["sliced"]) & set(open_vars)
        qt.qt_prepare(h, 0, 2)
        st = qt.qt_stats(h)
        assert st["n_open"] == len(opens)
        tot, steps = ledger.ledger([l for l, _ in tensors], plan["order"], plan["sliced"],
                                   plan["slice_step"])
        for key in ("prefix_flops", "slice_flops", "slice_bytes", "n_slice_steps"):
            assert st[key] == tot[key], key
        groups = ledger.launch_groups([l for l, _ in tensors], plan["order"], plan["sliced"],
                                      plan["slice_step"])
        assert st["groups"] == groups
        # back to one amplitude: the plain network again
        qt.qt_set_open(h, [])
        assert qt.qt_num_tensors(h)[1] == n * p
        with pytest.raises(qt.QtError) as e:
            qt.qt_prepare(h, 0, 1)
        assert e.value.status == qt.QT_ESTATE
    finally:
        qt.qt_free(h)


@pytest.mark.parametrize("n,p,seed,tau,q,rs", [(10, 2, 3, 1.0, 4, 11), (24, 2, 15, 0.5, 3, 12),
                                                 (30, 3, 11, 2.0, 2, 13), (44, 2, 14, 0.25, 5, 14),
                                                 (12, 1, 5, 1e-3, 3, 15), (12, 1, 5, 1e9, 3, 16)])
def test_rgreedy_bit_exact(qt, n, p, seed, tau, q, rs):
    """rgreedy (Sec. V.A.2): the library's order and widths equal the oracle's for the same
    seed of the draw stream."""
    from oracle import rgreedy
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    o, w, _ = rgreedy.rgreedy_order(adj, tau, q, rs)
    h = qt.qt_build_network(edges, n, p, gammas, betas, z)
    try:
        assert qt.qt_order_rgreedy(h, tau, q, rs) == max(w)
        assert qt.qt_get_order(h) == o and qt.qt_get_widths(h) == w
        with pytest.raises(qt.QtError) as e:
            qt.qt_order_rgreedy(h, 0.0, 1, 0)
        assert e.value.status == qt.QT_EINVAL
    finally:
        qt.qt_free(h)


def test_open_errors(qt):
    QtError = qt.QtError
    h = qt.qt_build_network([(0, 1), (1, 2)], 3, 1, [0.1], [0.2], [0, 1, 0])
    try:
        for bad in ([0, 0], [3], [-1], list(range(17))):
            with pytest.raises(QtError) as e:
                qt.qt_set_open(h, bad)
            assert e.value.status == qt.QT_EINVAL
        qt.qt_set_open(h, [2, 0])
        qt.qt_order(h, 0)
        qt.qt_prepare(h, 0, 1)
        # a single-amplitude call on a batched network is refused before any CUDA call
        with pytest.raises(QtError) as e:
            qt.qt_contract(h, 0, 256, 1 << 20, 0)
        assert e.value.status == qt.QT_ESTATE
        with pytest.raises(QtError) as e:
            qt.qt_contract_static(h, 0, 0)
        assert e.value.status == qt.QT_ESTATE
    finally:
        qt.qt_free(h)


def test_fusion_option(qt):
    """Without fusion every bucket is its own launch; with it, launch bytes only drop."""
    n, p, seed = 44, 2, 14
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    h = qt.qt_build_network(edges, n, p, gammas, betas, z)
    try:
        qt.qt_order(h, 0)
        qt.qt_slice(h, 17, 6, 1)
        qt.qt_prepare(h, 0, 2)
        fused = qt.qt_stats(h)
        qt.qt_set_option(h, qt.QT_OPT_FUSION, 0)
        with pytest.raises(qt.QtError):
            qt.qt_stats(h)  # the option discards the prepared schedule
        qt.qt_prepare(h, 0, 2)
        plain = qt.qt_stats(h)
        assert plain["fused"] == 0 and fused["fused"] == 1
        assert len(plain["groups"]) == len(plain["steps"])
        assert all(g[2] == 1 and g[5] == 1 for g in plain["groups"])
        assert plain["slice_launch_bytes"] == plain["slice_bytes"]
        assert fused["slice_launch_bytes"] < plain["slice_launch_bytes"]
        assert fused["slice_flops"] == plain["slice_flops"]
        with pytest.raises(qt.QtError):
            qt.qt_set_option(h, 99, 1)
    finally:
        qt.qt_free(h)


def test_set_angles_keeps_plan(qt):
    n, p, seed = 12, 2, 3
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    h = qt.qt_build_network(edges, n, p, gammas, betas, z)
    try:
        qt.qt_order(h, 0)
        qt.qt_slice(h, 6, 3, 1)
        before = (qt.qt_get_order(h), qt.qt_get_slices(h))
        qt.qt_prepare(h, 0, 2)
        qt.qt_set_angles(h, [0.5, 0.6], [0.7, 0.8])
        assert (qt.qt_get_order(h), qt.qt_get_slices(h)) == before
        qt.qt_stats(h)  # schedule still valid
    finally:
        qt.qt_free(h)


@pytest.mark.parametrize("n,p,seed,algo", [(16, 1, 3, 0), (16, 2, 3, 1), (12, 3, 5, 0),
                                           (40, 2, 9, 0)])
def test_energy_lightcone_orders_bit_exact(qt, n, p, seed, algo):
    """Every edge's lightcone network: variable count, greedy order and width equal the
    oracle's (same gate set, same variable numbering, same greedy rule)."""
    from oracle import energy, network, ordering
    from paper_2012_02430_gb300.inputs import qaoa_instance
    edges, g, b, z = qaoa_instance(n, p, seed)
    h = qt.qt_energy_build(edges, n, p, g, b, algo)
    try:
        for e, (u, v) in enumerate(edges):
            tensors, nv, norm = energy.lightcone_network(n, edges, p, g, b, u, v)
            adj = ordering.adjacency_matrix(network.line_graph(tensors, nv), nv)
            o, w = ordering.greedy_order(adj, None, {0: ordering.MIN_FILL, 1: ordering.MIN_DEGREE}[algo])
            assert qt.qt_energy_get_order(h, e) == (o, nv, max(w)), e
        qt.qt_energy_prepare(h, 0)
        st = qt.qt_energy_stats(h)
        assert st["edges"] == len(edges) and st["workspace_bytes"] > 0
    finally:
        qt.qt_energy_free(h)


def test_energy_sweep_errors(qt):
    """Angle sweeps refuse to run before qt_energy_prepare (no CUDA call is made)."""
    import ctypes as C
    h = qt.qt_energy_build([(0, 1), (1, 2), (2, 0)], 3, 1, [0.1], [0.2])
    try:
        need = C.c_size_t()
        assert qt.lib.qt_energy_sweep_prepare(h, 2, C.byref(need)) == qt.QT_ESTATE
        g = (C.c_double * 2)(0.1, 0.2)
        assert qt.lib.qt_energy_sweep(h, 2, g, g, None, 0, None, None, None) == qt.QT_EINVAL
    finally:
        qt.qt_energy_free(h)


def test_energy_errors(qt):
    with pytest.raises(qt.QtError) as e:
        qt.qt_energy_build([(0, 1), (1, 1)], 3, 1, [0.1], [0.2])
    assert e.value.status == qt.QT_EINVAL
    with pytest.raises(qt.QtError) as e:
        qt.qt_energy_build([(0, 1)], 2, 1, [0.1], [0.2], 5)
    assert e.value.status == qt.QT_EINVAL
    h = qt.qt_energy_build([(0, 1), (1, 2)], 3, 1, [0.1], [0.2])
    try:
        with pytest.raises(qt.QtError) as e:
            qt.qt_energy_stats(h)
        assert e.value.status == qt.QT_ESTATE
        with pytest.raises(qt.QtError) as e:
            qt.qt_energy_get_order(h, 7)
        assert e.value.status == qt.QT_EINVAL
    finally:
        qt.qt_energy_free(h)


@pytest.mark.parametrize("n,p,seed", [(20, 2, 3), (40, 2, 9), (30, 3, 4)])
def test_proposal_dataset_matches_oracle(qt, n, p, seed):
    """Features (float tolerance), labels and (s, v, width) bit-exact against the oracle."""
    import numpy as np
    from oracle import proposal
    from paper_2012_02430_gb300 import learn
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    X, Y, M = learn.dataset_of(edges, n, p, gammas, betas, z, topv=3)
    F, L, meta = proposal.dataset(adj, 0, 3)
    assert X.shape == F.shape
    assert np.max(np.abs(X - F)) <= 1e-6
    assert [tuple(r) for r in M] == [tuple(r) for r in meta]
    assert np.max(np.abs(Y - L)) <= 1e-6


@pytest.mark.parametrize("case", [(12, 3, 3, 8, 4, 1), (24, 3, 15, 14, 6, 2), (40, 2, 9, 11, 4, 1)])
def test_learned_search_without_model_is_the_papers(qt, case):
    """qt_slice_learned with no model, topv = 1 and an unlimited spread is qt_slice's search."""
    import ctypes as C
    n, p, seed, lim, mv, r = case
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    plan = oracle_plan(adj, 0, lim, mv, r)
    h = qt.qt_build_network(edges, n, p, gammas, betas, z)
    try:
        qt.qt_order(h, 0)
        k, w = C.c_int32(), C.c_int32()
        qt._check(qt.lib.qt_slice_learned(h, None, 64, lim, mv, r, 1, 0, 1 << 30, C.byref(k),
                                          C.byref(w)))
        assert qt.qt_get_slices(h) == (plan["sliced"], plan["slice_step"])
        assert qt.qt_get_order(h) == plan["order"] and w.value == plan["width"]
        runs = C.c_int64()
        qt._check(qt.lib.qt_plan_info(h, C.byref(runs), None))
        qt.qt_order(h, 0)
        qt.qt_slice(h, lim, mv, r)
        runs2 = C.c_int64()
        qt._check(qt.lib.qt_plan_info(h, C.byref(runs2), None))
        assert runs.value == runs2.value
    finally:
        qt.qt_free(h)


def test_mlp_forward_host_matches_oracle(qt):
    import ctypes as C
    import numpy as np
    from oracle import mlp
    nf, hidden, batch = 16, 24, 11
    rng = np.random.default_rng(7)
    p = rng.normal(0, 0.4, mlp.n_params(nf, hidden)).astype(np.float32)
    x = rng.normal(0, 1, (batch, nf)).astype(np.float32)
    y = np.zeros(batch, dtype=np.float32)
    fp = C.POINTER(C.c_float)
    qt._check(qt.lib.qt_mlp_forward_host(p.ctypes.data_as(fp), nf, hidden, x.ctypes.data_as(fp),
                                         batch, y.ctypes.data_as(fp)))
    ref, _ = mlp.forward(p.astype(np.float64), x.astype(np.float64), nf, hidden)
    assert np.max(np.abs(y - ref)) <= 1e-5 * max(1.0, np.max(np.abs(ref)))


def test_mlp_forward_host_hand_example(qt):
    """The library's host forward on the hand-worked 2-3-3-1 example (values exact in FP32)."""
    import ctypes as C
    import json
    import numpy as np
    with open(os.path.join(ROOT, "tests", "golden", "mlp_hand.json")) as f:
        g = json.load(f)
    p = np.concatenate([np.ravel(g["W1"]), g["b1"], np.ravel(g["W2"]), g["b2"], g["w3"],
                        [g["b3"]]]).astype(np.float32)
    x = np.array(g["x"], dtype=np.float32)
    y = np.zeros(len(x), dtype=np.float32)
    fp = C.POINTER(C.c_float)
    qt._check(qt.lib.qt_mlp_forward_host(p.ctypes.data_as(fp), g["nf"], g["hidden"],
                                         x.ctypes.data_as(fp), len(x), y.ctypes.data_as(fp)))
    assert y.tolist() == g["y"]


def test_segment_option_range(qt):
    """QT_OPT_SEGMENTS takes 0 (off), 1 (on, default limit) or a limit of 2..13 union
    indices; other values are refused."""
    net = qt.Network([(0, 1), (1, 2), (2, 0)], 3, 1, [0.3], [0.2], [0, 1, 0])
    for v in (0, 1, 2, 12, 13):
        qt.qt_set_option(net.handle, qt.QT_OPT_SEGMENTS, v)
    for v in (-1, 14, 1 << 40):
        with pytest.raises(qt.QtError):
            qt.qt_set_option(net.handle, qt.QT_OPT_SEGMENTS, v)


def test_gemm_option_range(qt):
    """QT_OPT_GEMM takes 0, 1 (the GEMM form by default) or 2 (with the streaming kernel
    where it applies); other values are refused."""
    net = qt.Network([(0, 1), (1, 2), (2, 0)], 3, 1, [0.3], [0.2], [0, 1, 0])
    for v in (0, 1, 2):
        qt.qt_set_option(net.handle, qt.QT_OPT_GEMM, v)
    for v in (-1, 3):
        with pytest.raises(qt.QtError):
            qt.qt_set_option(net.handle, qt.QT_OPT_GEMM, v)


def test_tma_option_range(qt):
    """QT_OPT_TMA takes 0..4 (off, on, and on with a fixed register block); other values
    are refused."""
    net = qt.Network([(0, 1), (1, 2), (2, 0)], 3, 1, [0.3], [0.2], [0, 1, 0])
    for v in range(5):
        qt.qt_set_option(net.handle, qt.QT_OPT_TMA, v)
    for v in (-1, 5):
        with pytest.raises(qt.QtError):
            qt.qt_set_option(net.handle, qt.QT_OPT_TMA, v)


def test_set_angles_rewrites_tensors_in_place(qt):
    """qt_set_angles rewrites the network's tensors in place: after new angles (also with
    open qubits, and after a new bitstring) every tensor's labels and values equal those of
    a network built with those angles and that bitstring from the start, bit for bit."""
    from paper_2012_02430_gb300.inputs import qaoa_instance, random_angles, random_bitstring
    edges, g, b, z = qaoa_instance(20, 3, 77)
    for open_q in ([], [3, 11]):
        net = qt.qt_build_network(edges, 20, 3, g, b, z)
        try:
            if open_q:
                qt.qt_set_open(net, open_q)
            for i in range(3):
                g2, b2 = random_angles(3, 900 + i)
                z2 = random_bitstring(20, 950 + i) if i == 2 else z
                if i == 2:
                    qt.qt_set_bitstring(net, z2)
                qt.qt_set_angles(net, g2, b2)
                ref = qt.qt_build_network(edges, 20, 3, g2, b2, z2)
                try:
                    if open_q:
                        qt.qt_set_open(ref, open_q)
                    cnt, nv = qt.qt_num_tensors(net)
                    assert (cnt, nv) == qt.qt_num_tensors(ref)
                    for t in range(cnt):
                        assert qt.qt_get_tensor(net, t) == qt.qt_get_tensor(ref, t), (open_q, i, t)
                finally:
                    qt.qt_free(ref)
        finally:
            qt.qt_free(net)


def test_seg_cluster_and_tcgen05_option_ranges(qt):
    """QT_OPT_SEG_CLUSTER takes 0 (chosen per launch) or a cluster size of 1, 2, 4 or 8;
    QT_OPT_TCGEN05 takes 0..4 (4: every tcgen05 work unit carries 4 summed values); other
    values are refused with QT_EINVAL."""
    net = qt.Network([(0, 1), (1, 2), (2, 0)], 3, 1, [0.3], [0.2], [0, 1, 0])
    for v in (0, 1, 2, 4, 8):
        qt.qt_set_option(net.handle, qt.QT_OPT_SEG_CLUSTER, v)
    for v in (-1, 3, 5, 16):
        with pytest.raises(qt.QtError) as e:
            qt.qt_set_option(net.handle, qt.QT_OPT_SEG_CLUSTER, v)
        assert e.value.status == qt.QT_EINVAL
    for v in range(5):
        qt.qt_set_option(net.handle, qt.QT_OPT_TCGEN05, v)
    for v in (-1, 5):
        with pytest.raises(qt.QtError) as e:
            qt.qt_set_option(net.handle, qt.QT_OPT_TCGEN05, v)
        assert e.value.status == qt.QT_EINVAL


def test_tensor_regions_aligned(qt):
    """The prefix and slice regions of the workspace start on 1024 bytes, so tensor offsets
    aligned to 64 elements inside them are aligned in the workspace: every per-slice operand
    of a GEMM-form launch (the slice region) has its rows of up to 64 summed values start on
    a row boundary. (Gates are packed two-element aligned and are not checked.)"""
    from paper_2012_02430_gb300.inputs import qaoa_instance
    for n, p, seed, wl, prec in ((120, 3, 1003, 28, 3), (80, 2, 1002, 26, 0), (30, 3, 7, 0, 4)):
        edges, g, b, z = qaoa_instance(n, p, seed)
        net = qt.Network(edges, n, p, g, b, z)
        net.order(0)
        if wl:
            net.slice(wl, 43, 1)
        qt.qt_prepare(net.handle, prec, 2)
        for L in qt.qt_launch_plan(net.handle)["launches"]:
            gm = L.get("gemm")
            if not gm:
                continue
            K = 1 << gm["nsum"]
            for side in ("A", "B"):
                base, stride, smask, sshift = gm[side]
                if stride:
                    assert base % min(K, 64) == 0 and stride % min(K, 64) == 0, (n, gm["step"], side)


def test_contract_sweep_errors(qt):
    """qt_contract_sweep refuses bad arguments before any device work: no sets, a non-finite
    angle, a network that is not ordered, or one with open qubits."""
    import ctypes as C
    lib = qt.lib
    net = qt.Network([(0, 1), (1, 2), (2, 0)], 3, 1, [0.3], [0.2], [0, 1, 0])
    out = (C.c_double * 4)()
    g = (C.c_double * 2)(0.1, 0.2)
    b = (C.c_double * 2)(0.3, 0.4)
    assert lib.qt_contract_sweep(net.handle, 0, 2, g, b, None, 0, None, out) == qt.QT_ESTATE
    net.order(0)
    assert lib.qt_contract_sweep(net.handle, 0, 0, g, b, None, 0, None, out) == qt.QT_EINVAL
    assert lib.qt_contract_sweep(net.handle, 0, 2, None, b, None, 0, None, out) == qt.QT_EINVAL
    bad = (C.c_double * 2)(0.1, float("nan"))
    assert lib.qt_contract_sweep(net.handle, 0, 2, bad, b, None, 0, None, out) == qt.QT_EINVAL
    net.set_open([0])
    assert lib.qt_contract_sweep(net.handle, 0, 2, g, b, None, 0, None, out) == qt.QT_ESTATE


@pytest.mark.parametrize("case", [(80, 2, 1002, 26, 20), (50, 3, 1003, 28, 20), (32, 3, 25, 0, 0)])
def test_launch_form_masks(qt, case):
    """The schedule's GEMM-form and triangle-form classifications are exact set relations
    over each launch's union U: GEMM form -- summed-in-both (K) and batch indices lie in
    A and B, A-only outputs in A and not B, B-only outputs in B and not A, one-sided summed
    indices in one side only, the six classes disjoint and covering U; triangle form --
    K in A and B only, X in A and C only, Y in B and C only, and every summed index of U
    in exactly one class."""
    n, p, seed, wl, mv = case
    from paper_2012_02430_gb300.inputs import qaoa_instance
    edges, g, b, z = qaoa_instance(n, p, seed)
    net = qt.Network(edges, n, p, g, b, z)
    qt.qt_set_option(net.handle, qt.QT_OPT_TRIANGLE, 1)
    net.order(0)
    if wl:
        net.slice(wl, mv, 1)
    qt.qt_prepare(net.handle, 0, 1)
    st = net.stats()
    assert st["gemm_masks"] and (st["tri_masks"] or n == 50)  # both forms are exercised
    for first, u, mK, mSA, mSB, mM, mN, mBt, uA, uB, na, nb in st["gemm_masks"]:
        full = (1 << u) - 1
        classes = [mK, mSA, mSB, mM, mN, mBt]
        assert sum(bin(c).count("1") for c in classes) == u, first
        acc = 0
        for c in classes:
            assert c & acc == 0, first
            acc |= c
        assert acc == full, first
        assert mK & ~(uA & uB) == 0 and mBt & ~(uA & uB) == 0, first
        assert mM & ~(uA & ~uB) == 0 and mSA & ~(uA & ~uB) == 0, first
        assert mN & ~(uB & ~uA) == 0 and mSB & ~(uB & ~uA) == 0, first
        assert na >= 1 and nb >= 1, first
    for first, u, tK, tX, tY, uA, uB, uC in st["tri_masks"]:
        assert tK & tX == 0 and tK & tY == 0 and tX & tY == 0, first
        assert tK & ~(uA & uB & ~uC) == 0, first
        assert tX & ~(uA & uC & ~uB) == 0, first
        assert tY & ~(uB & uC & ~uA) == 0, first
        nsum = bin(tK | tX | tY).count("1")
        assert tK | tX | tY == (1 << nsum) - 1, first  # the summed indices are U's lowest


def _plan_reaches(plan):
    """reach[m] = the set of launches that launch m is ordered after: the earlier launches
    on its stream and, through waits, everything those and the waited-for launches follow."""
    launches = plan["launches"]
    reach = []
    last_on = {}
    for m, d in enumerate(launches):
        before = set()
        prev = last_on.get(d["stream"])
        if prev is not None:
            before |= {prev} | reach[prev]
        for w in d["wait"]:
            assert 0 <= w < m and launches[w]["stream"] != d["stream"]
            before |= {w} | reach[w]
        reach.append(before)
        last_on[d["stream"]] = m
    return reach


@pytest.mark.parametrize("case", [(80, 2, 1002, 26, 20, 4), (44, 2, 14, 0, 0, 1),
                                  (60, 2, 18, 23, 6, 4), (50, 3, 1003, 28, 20, 2)])
def test_launch_plan_orders_every_conflict(qt, case):
    """The concurrent plan of the slice phase: any two launches where one writes arena
    elements the other reads or writes are ordered (same stream, or a chain of waits),
    streams are in range, and every launch's ranges are well formed."""
    n, p, seed, wl, mv, batch = case
    from paper_2012_02430_gb300.inputs import qaoa_instance
    edges, g, b, z = qaoa_instance(n, p, seed)
    net = qt.Network(edges, n, p, g, b, z)
    net.order(0)
    if wl:
        net.slice(wl, mv, 1)
    qt.qt_prepare(net.handle, 0, batch)
    plan = qt.qt_launch_plan(net.handle)
    launches = plan["launches"]
    assert launches and all(0 <= d["stream"] < plan["streams"] for d in launches)
    for d in launches:
        for lo, hi in d["reads"] + d["writes"]:
            assert 0 <= lo < hi
    reach = _plan_reaches(plan)

    def meet(xs, ys):
        return any(a < d and c < b for a, b in xs for c, d in ys)

    conflicts = 0
    for m, dm in enumerate(launches):
        for l in range(m):
            dl = launches[l]
            if (meet(dl["writes"], dm["reads"]) or meet(dl["writes"], dm["writes"])
                    or meet(dl["reads"], dm["writes"])):
                conflicts += 1
                assert l in reach[m], (l, m)
    assert conflicts > 0
    # more than one stream carries work on the larger plans
    if n >= 60:
        assert len({d["stream"] for d in launches}) > 1


@pytest.mark.parametrize("case", [(80, 2, 1002, 26, 20, 4), (60, 2, 18, 23, 6, 4),
                                  (50, 3, 1003, 28, 20, 2), (24, 3, 15, 0, 0, 4)])
def test_segment_work_items(qt, case):
    """Segment launches (host planning, no GPU): every step of a level is cut into work
    items of 32 value pairs, max(1, 2^(u-1) / 32) of them, the level's item count is their
    sum, the levels hold every step once, no step sums more than 6 indices (the shuffle
    reduction stays inside a warp) or exceeds the segment's union limit, and the largest
    cluster the device co-schedules is 1 without a GPU."""
    n, p, seed, wl, mv, batch = case
    from paper_2012_02430_gb300.inputs import qaoa_instance
    edges, g, b, z = qaoa_instance(n, p, seed)
    net = qt.Network(edges, n, p, g, b, z)
    net.order(0)
    if wl:
        net.slice(wl, mv, 1)
    qt.qt_prepare(net.handle, 0, batch)
    segs = [L["segment"] for L in qt.qt_launch_plan(net.handle)["launches"] if "segment" in L]
    assert segs
    for sg in segs:
        steps, levels = sg["steps"], sg["levels"]
        assert sum(nw + nb for nw, nb, _ in levels) == len(steps) >= 2
        first = 0
        for nw, nb, items in levels:
            lv = steps[first:first + nw + nb]
            assert all(u <= 6 for _, u, _ in lv[:nw])  # warp steps: at most 32 value pairs
            assert items == sum(max(1, (1 << (u - 1)) // 32) for _, u, _ in lv)
            first += nw + nb
        assert all(1 <= m <= 12 and 1 <= nsum <= 6 and nsum <= u <= 12 for m, u, nsum in steps)
        assert sg["arena"] > 0 and sg["cluster_max"] in (1, 2, 4, 8)


UMMA_PLAN_CASES = [(30, 3, 5, -4), (44, 2, 3, -2), (60, 2, 19, -4), (50, 2, 7, -2),
                   (48, 2, 5, 0), (44, 3, 15, -2), (50, 2, 22, -4), (24, 3, 21, 0),
                   (80, 2, 1002, 26 - 35)]


@pytest.mark.parametrize("case", UMMA_PLAN_CASES)
def test_tcgen05_plan_invariants(qt, case):
    """The tcgen05 GEMM's tiling of each launch it takes (host planning, no GPU): 128 lanes
    from the 7 lowest only-indices of one side, at least 8 columns from the other side,
    group indices among the batch indices, every output index in exactly one of lanes,
    columns, group and tile indices; the tile covers a prefix of the output indices as
    long as tensor memory allows; an epilogue chunk's runs start at output bit 0; the
    unit boxes' row runs add up to the lanes and columns; tensor and shared memory in
    range."""
    n, p, seed, off = case
    edges, gammas, betas, z, *_ = oracle_problem(n, p, seed)
    h = qt.qt_build_network(edges, n, p, gammas, betas, z)
    try:
        qt.qt_set_option(h, qt.QT_OPT_TCGEN05, 1)
        w = qt.qt_order(h, 0)
        if off:
            qt.qt_slice(h, w + off, 20 if n == 80 else 6, 1)
        qt.qt_prepare(h, 3, 2)
        plans = [L["umma"] for L in qt.qt_launch_plan(h)["launches"] if "umma" in L]
    finally:
        qt.qt_free(h)
    assert plans
    pop = lambda m: bin(m).count("1")
    for u in plans:
        ns = u["nsum"]
        assert u["mK"] == (1 << ns) - 1 and 2 <= ns <= 6
        lonly, conly = (u["mM"], u["mN"]) if u["lside"] == 0 else (u["mN"], u["mM"])
        lowest = lambda m, k: sum(1 << b for b in sorted(b for b in range(32) if m >> b & 1)[:k])
        assert pop(u["mlane"]) == 7 and u["mlane"] == lowest(lonly, 7)
        assert u["mcol"] & ~conly == 0 and pop(u["mcol"]) == u["cb"] and 3 <= u["cb"] <= 7
        assert u["mgrp"] & ~u["mBt"] == 0 and pop(u["mgrp"]) == u["gb"] <= 4
        out_bits = (u["mM"] | u["mN"] | u["mBt"]) & ~((1 << ns) - 1)
        rest = sum(1 << b for b in u["rest"])
        parts = [u["mlane"], u["mcol"], u["mgrp"], rest]
        assert sum(pop(x) for x in parts) == pop(out_bits)
        assert parts[0] | parts[1] | parts[2] | parts[3] == out_bits
        tile = u["mlane"] | u["mcol"] | u["mgrp"]
        # the covered prefix: output bits ns .. ns + prefix - 1 all belong to the tile
        assert u["prefix"] >= 1 and all(tile >> b & 1 for b in range(ns, ns + u["prefix"]))
        G, Nt = 1 << u["gb"], 1 << u["cb"]
        assert G * Nt <= 128
        cols = u["tmem_cols"]
        assert cols & (cols - 1) == 0 and 4 * G * Nt <= cols <= 512
        # epilogue chunk: lanes 0-4, the groups and the lowest 2^cwb columns, in output bits
        chunk = (lowest(u["mlane"], 5) | u["mgrp"] | lowest(u["mcol"], u["cwb"])) >> ns
        assert u["chunk_out"] == chunk and pop(chunk) == 5 + u["gb"] + u["cwb"] <= 10
        assert u["rb"] >= 1 and chunk & ((1 << u["rb"]) - 1) == (1 << u["rb"]) - 1
        assert not (chunk >> u["rb"]) & 1
        assert sum(l for _, l in u["lruns"]) == 7 and sum(l for _, l in u["cruns"]) == u["cb"]
        assert 1 <= len(u["lruns"]) <= 3 and 1 <= len(u["cruns"]) <= 3
        assert u["smem"] <= 225 * 1024 and u["passes"] == 3
        assert 2 <= u["sraw"] <= 8 and 1 <= u["splane"] <= 4
        assert 2 <= u["kc"] <= ns


def test_tcgen05_chunks_long_rows(qt):
    """N=120, p=3, seed 1003 sliced to rank 28 (the many-slice workload), split TF32:
    the launches with 6 summed indices (rows of 64 complex) take the tcgen05 form with
    chunks of the summed values, 4 raw units and 2 plane slots in flight; launches whose
    rows fit whole keep them whole."""
    from paper_2012_02430_gb300.inputs import qaoa_instance
    edges, g, b, z = qaoa_instance(120, 3, 1003)
    net = qt.Network(edges, 120, 3, g, b, z)
    net.order(0)
    net.slice(28, 43, 1)
    qt.qt_prepare(net.handle, 3, 266)
    plans = [L["umma"] for L in qt.qt_launch_plan(net.handle)["launches"] if "umma" in L]
    deep = [u for u in plans if u["nsum"] == 6]
    assert len(deep) >= 2
    for u in deep:
        assert 2 <= u["kc"] < 6 and u["sraw"] >= 4 and u["splane"] >= 2
        assert u["smem"] <= 225 * 1024
    assert all(u["kc"] == u["nsum"] for u in plans if u["nsum"] <= 3)


@pytest.mark.parametrize("case", [(12, 1, 3, 0), (16, 2, 5, 0), (14, 2, 9, 1)])
def test_order_dataset_matches_oracle(qt, case):
    """qt_order_dataset (elimination-step candidates, features, rollout labels) against the
    oracle's restatement: candidates and rollout widths bit-exact, features and labels to
    FP32 rounding."""
    import ctypes as C
    import numpy as np
    from oracle import ordering, proposal
    n, p, seed, algo = case
    edges, gammas, betas, z, tensors, nv, norm, adj = oracle_problem(n, p, seed)
    h = qt.qt_build_network(edges, n, p, gammas, betas, z)
    try:
        qt.qt_order(h, algo)
        cnt = C.c_int32()
        qt._check(qt.lib.qt_order_dataset(h, 4, 3, None, None, None, 0, C.byref(cnt)))
        k = cnt.value
        f = (C.c_float * (k * 16))()
        lab = (C.c_float * k)()
        meta = (C.c_int32 * (3 * k))()
        qt._check(qt.lib.qt_order_dataset(h, 4, 3, f, lab, meta, k, C.byref(cnt)))
    finally:
        qt.qt_free(h)
    X = np.frombuffer(f, dtype=np.float32).reshape(k, 16)
    L = np.frombuffer(lab, dtype=np.float32)
    M = np.frombuffer(meta, dtype=np.int32).reshape(k, 3)
    rule = ordering.MIN_DEGREE if algo else ordering.MIN_FILL
    Xo, Lo, Mo = proposal.order_dataset(adj, rule, 4, 3)
    assert [tuple(int(x) for x in m) for m in M] == [tuple(m) for m in Mo]
    assert np.allclose(X, Xo, rtol=1e-6, atol=1e-6)
    assert np.allclose(L, Lo, rtol=1e-6, atol=1e-6)
