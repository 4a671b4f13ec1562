"""The FP64 oracle against what the paper and the mathematics fix (no GPU).

Pins: the 2^N statevector (brute force), closed forms at gamma = 0 and beta = 0,
normalisation, the closed-form p=1 MaxCut edge energy (Wang et al.), numpy's
own einsum over the whole network, hand-worked greedy and slicing examples
(tests/golden), the slice-sum invariant (Eq. 2), brute-force minimum width on
tiny graphs, and numbers printed in the paper for the ledger's conventions.
"""

import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import contract, energy, ledger, network, ordering, rgreedy, slicing, statevector
from paper_2012_02430_gb300.inputs import qaoa_instance, random_regular_graph

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def adj_of(n, edges):
    a = np.zeros((n, n), dtype=bool)
    for u, v in edges:
        a[u, v] = a[v, u] = True
    return a


def problem(n, p, seed):
    edges, g, b, z = qaoa_instance(n, p, seed)
    t, nv, norm = network.build_network(n, edges, p, g, b, z)
    adj = ordering.adjacency_matrix(network.line_graph(t, nv), nv)
    return edges, g, b, z, t, nv, norm, adj


# ----------------------------- network & statevector ------------------------

def test_gate_matrices_match_matrix_exponentials():
    from scipy.linalg import expm
    x = np.array([[0, 1], [1, 0]], dtype=complex)
    for beta in (0.0, 0.37, 1.9, 3.0):
        u = expm(-1j * beta * x)  # exp(-i beta X), rows a', columns a
        m = network.mixer_matrix(beta)  # M[a, a'] = <a'|U|a>
        assert np.allclose(m, u.T, atol=1e-14)
    zz = np.diag([1, -1, -1, 1]).astype(complex)
    for gamma in (0.0, 0.5, 2.2):
        cost = expm(-1j * gamma * 0.5 * (np.eye(4) - zz))
        d = network.phase_matrix(gamma)
        assert np.allclose(np.diag(cost).reshape(2, 2), d, atol=1e-14)


def test_network_counts():
    n, p = 10, 3
    edges, g, b, z = qaoa_instance(n, p, 4)
    t, nv, norm = network.build_network(n, edges, p, g, b, z)
    assert nv == n * p
    assert len(t) == n + p * len(edges) + n * (p - 1) + n
    assert norm == 2.0 ** (-n / 2)


def test_random_regular_graph_is_simple_and_regular():
    for n, seed in [(10, 1), (80, 1002), (210, 1005)]:
        e = random_regular_graph(n, 3, seed)
        assert len(e) == 3 * n // 2 and len(set(e)) == len(e)
        deg = [0] * n
        for u, v in e:
            assert u < v
            deg[u] += 1
            deg[v] += 1
        assert deg == [3] * n


@pytest.mark.parametrize("n,p,seed", [(6, 1, 1), (8, 2, 2), (10, 3, 3)])
def test_statevector_normalised(n, p, seed):
    edges, g, b, z = qaoa_instance(n, p, seed)
    psi = statevector.qaoa_state(n, edges, g, b)
    assert abs(np.vdot(psi, psi) - 1) < 1e-12


def test_statevector_mixer_matches_full_exponential():
    """The per-qubit mixer equals exp(-i beta sum_v X_v) built as one 2^N matrix."""
    from scipy.linalg import expm
    n = 4
    edges = [(0, 1), (1, 2), (2, 3), (0, 3)]
    g, b = [0.8], [0.45]
    x = np.array([[0, 1], [1, 0]], dtype=complex)
    bsum = np.zeros((1 << n, 1 << n), dtype=complex)
    for q in range(n):
        ops = [np.eye(2)] * n
        ops[n - 1 - q] = x  # kron order: qubit q is bit q of the index
        m = ops[0]
        for o in ops[1:]:
            m = np.kron(m, o)
        bsum += m
    cut = statevector.cut_values(n, edges)
    psi0 = np.full(1 << n, 2 ** (-n / 2), dtype=complex)
    ref = expm(-1j * b[0] * bsum) @ (np.exp(-1j * g[0] * cut) * psi0)
    assert np.allclose(statevector.qaoa_state(n, edges, g, b), ref, atol=1e-13)


@pytest.mark.parametrize("n,p,seed", [(8, 1, 11), (10, 2, 12), (12, 3, 13)])
def test_closed_forms_gamma_zero_beta_zero(n, p, seed):
    edges, g, b, z = qaoa_instance(n, p, seed)
    t, nv, norm = network.build_network(n, edges, p, [0.0] * p, b, z)
    adj = ordering.adjacency_matrix(network.line_graph(t, nv), nv)
    o, _ = ordering.greedy_order(adj)
    a, _ = contract.contract_amplitude(t, o)
    assert abs(a * norm - 2 ** (-n / 2) * np.exp(-1j * n * sum(b))) < 1e-13
    t, nv, norm = network.build_network(n, edges, p, g, [0.0] * p, z)
    a, _ = contract.contract_amplitude(t, o)
    cut = sum(z[u] != z[v] for u, v in edges)
    assert abs(a * norm - 2 ** (-n / 2) * np.exp(-1j * sum(g) * cut)) < 1e-13


# ----------------------------- bucket elimination ---------------------------

@pytest.mark.parametrize("n,p,seed,algo", [(6, 1, 21, 0), (10, 2, 22, 1), (12, 3, 23, 0),
                                           (14, 2, 24, 1), (20, 1, 1001, 0)])
def test_bucket_elimination_equals_statevector(n, p, seed, algo):
    edges, g, b, z, t, nv, norm, adj = problem(n, p, seed)
    o, _ = ordering.greedy_order(adj, None, algo)
    a, _ = contract.contract_amplitude(t, o)
    sv = statevector.amplitude(n, edges, g, b, z)
    assert abs(a * norm - sv) <= 1e-12 * abs(sv)


def test_bucket_elimination_equals_whole_network_einsum():
    """numpy's einsum over the whole network, its own path: an independent contraction."""
    n, p = 6, 2
    edges, g, b, z, t, nv, norm, adj = problem(n, p, 31)
    args = []
    for labels, data in t:
        args += [data, list(labels)]
    whole = np.einsum(*args, [], optimize="greedy")
    o, _ = ordering.greedy_order(adj)
    a, _ = contract.contract_amplitude(t, o)
    assert abs(a - whole) < 1e-12 * abs(whole)


@pytest.mark.parametrize("n,p,seed,algo,drop,r", [(10, 2, 2, 0, 2, 1), (12, 3, 3, 1, 3, 2),
                                                  (16, 2, 41, 0, 3, 1), (14, 3, 42, 1, 4, 1)])
def test_slicing_sum_invariant(n, p, seed, algo, drop, r):
    """Eq. 2: the sum over all slices equals the unsliced contraction."""
    edges, g, b, z, t, nv, norm, adj = problem(n, p, seed)
    o, w = ordering.greedy_order(adj, None, algo)
    full, _ = contract.contract_amplitude(t, o)
    plan = slicing.step_dependent_slicing(adj, algo, max(w) - drop, 4, r)
    assert plan["sliced"], "the plan must slice"
    tot, per = contract.contract_amplitude(t, plan["order"], plan["sliced"], plan["slice_step"])
    assert len(per) == 1 << len(plan["sliced"])
    assert abs(tot - full) < 1e-12 * abs(full)
    sv = statevector.amplitude(n, edges, g, b, z)
    assert abs(tot * norm - sv) < 1e-12 * abs(sv)


# ----------------------------- randomised greedy (Sec. V.A.2) ---------------

def test_rgreedy_boltzmann_first_pick_frequencies():
    """Star K_{1,3}: leaves have degree 1, the centre 3. With tau = 1 the first vertex is
    the centre with probability e^-3 / (3 e^-1 + e^-3); over 20000 seeds the observed
    frequency is within 4 standard deviations (a sign or tau mistake fails this)."""
    star = adj_of(4, [(0, 1), (0, 2), (0, 3)])
    n = 20000
    hits = 0
    for seed in range(n):
        o, _, _ = rgreedy.rgreedy_order(star, 1.0, 1, seed)
        hits += o[0] == 0
    pc = math.exp(-3) / (3 * math.exp(-1) + math.exp(-3))
    sd = math.sqrt(pc * (1 - pc) / n)
    assert abs(hits / n - pc) < 4 * sd, (hits / n, pc)


def test_rgreedy_small_tau_is_min_degree():
    """tau -> 0 puts all the weight on the smallest degrees: every step takes a vertex of
    minimum current degree (the paper's greedy), ties broken at random."""
    edges, g, b, z, t, nv, norm, adj = problem(14, 2, 61)
    for seed in range(5):
        o, w, _ = rgreedy.rgreedy_order(adj, 1e-3, 1, seed)
        a = adj.copy()
        alive = np.ones(nv, dtype=bool)
        np.fill_diagonal(a, False)
        for v in o:
            degs = a[alive].sum(axis=1)
            assert a[v].sum() == degs.min()
            ordering.eliminate(a, alive, v)
        assert sorted(o) == list(range(nv))


def test_rgreedy_large_tau_is_uniform():
    """tau -> infinity: the first vertex is uniform over the vertices (chi-square)."""
    edges, g, b, z, t, nv, norm, adj = problem(8, 1, 62)
    counts = np.zeros(nv)
    n = 8000
    for seed in range(n):
        o, _, _ = rgreedy.rgreedy_order(adj, 1e12, 1, seed)
        counts[o[0]] += 1
    chi2 = ((counts - n / nv) ** 2 / (n / nv)).sum()
    assert chi2 < 30.0, chi2  # 7 degrees of freedom: p < 1e-4 above 30


def test_rgreedy_keeps_best_of_q_and_is_a_valid_order():
    edges, g, b, z, t, nv, norm, adj = problem(16, 2, 63)
    o, w, runs = rgreedy.rgreedy_order(adj, 0.5, 6, 7)
    assert sorted(o) == list(range(nv)) and max(w) == min(runs)
    assert ordering.replay_widths(adj, o) == w
    a, _ = contract.contract_amplitude(t, o)
    sv = statevector.amplitude(16, edges, g, b, z)
    assert abs(a * norm - sv) <= 1e-12 * abs(sv)


# ----------------------------- batch of amplitudes (Sec. VII) --------------

def open_problem(n, p, seed, opens):
    edges, g, b, z = qaoa_instance(n, p, seed)
    t, nv, norm = network.build_network(n, edges, p, g, b, z, opens)
    sets = network.open_clique(network.line_graph(t, nv), n, p, len(opens))
    adj = ordering.adjacency_matrix(sets, nv)
    keep = np.zeros(nv, dtype=bool)
    keep[n * p:] = True
    return edges, g, b, z, t, nv, norm, adj, keep


@pytest.mark.parametrize("n,p,seed,opens,algo,drop", [
    (8, 1, 51, [0], 0, 0), (10, 2, 52, [3, 7], 1, 0), (12, 2, 53, [11, 0, 5], 0, 2),
    (12, 3, 54, [2, 4, 6, 8], 0, 3), (14, 2, 55, [1, 9, 13], 1, 2)])
def test_open_batch_equals_statevector(n, p, seed, opens, algo, drop):
    """Entry b of the open contraction is the amplitude of z with the open qubits set to
    the bits of b (brute force over the 2^N statevector), sliced or not (Eq. 2)."""
    edges, g, b, z, t, nv, norm, adj, keep = open_problem(n, p, seed, opens)
    o, w = ordering.greedy_order(adj, None, algo, keep)
    assert not set(o) & set(range(n * p, nv))
    plan = slicing.step_dependent_slicing(adj, algo, max(w) - drop if drop else 1 << 30, 4, 1,
                                          keep)
    assert not set(plan["sliced"]) & set(range(n * p, nv))
    if drop:
        assert plan["sliced"], "the plan must slice"
    ov = list(range(n * p, nv))
    tot, per = contract.contract_amplitude(t, plan["order"], plan["sliced"], plan["slice_step"],
                                           open_vars=ov)
    psi = statevector.qaoa_state(n, edges, g, b)
    a = len(opens)
    for bits in range(1 << a):
        zz = list(z)
        for j, v in enumerate(opens):
            zz[v] = (bits >> j) & 1
        want = psi[sum(x << v for v, x in enumerate(zz))]
        got = tot[tuple((bits >> j) & 1 for j in range(a))] * norm
        assert abs(got - want) <= 1e-12 * max(abs(want), 1e-300) + 1e-15, bits


def test_open_batch_bits_of_z_at_open_qubits_are_ignored():
    n, p, seed, opens = 10, 2, 56, [4, 2]
    edges, g, b, z, t, nv, norm, adj, keep = open_problem(n, p, seed, opens)
    z2 = list(z)
    for v in opens:
        z2[v] ^= 1
    t2, _, _ = network.build_network(n, edges, p, g, b, z2, opens)
    o, _ = ordering.greedy_order(adj, None, 0, keep)
    a1, _ = contract.contract_amplitude(t, o, open_vars=list(range(n * p, nv)))
    a2, _ = contract.contract_amplitude(t2, o, open_vars=list(range(n * p, nv)))
    assert np.array_equal(a1, a2)


def test_open_greedy_hand_example():
    """Path 0-1-2 with vertex 1 kept: min-fill takes 0 (fill 0, degree 1), then 2 (its
    only neighbour is 1); vertex 1 is never eliminated. Without the mark: 0, 1, 2."""
    a = adj_of(3, [(0, 1), (1, 2)])
    keep = np.array([False, True, False])
    assert ordering.greedy_order(a, None, 0, keep) == ([0, 2], [1, 1])
    assert ordering.greedy_order(a, None, 0) == ([0, 1, 2], [1, 1, 0])
    # slicing never removes a kept vertex, even the one with most neighbours
    star = adj_of(4, [(0, 1), (0, 2), (0, 3), (1, 2)])
    keep = np.array([True, False, False, False])
    plan = slicing.step_dependent_slicing(star, 0, 1, 1, 1, keep)
    assert plan["sliced"] and 0 not in plan["sliced"] and 0 not in plan["order"]


# ----------------------------- orders and widths ----------------------------

def test_greedy_hand_examples():
    for c in load("greedy_hand.json")["cases"]:
        a = adj_of(c["n"], c["edges"])
        for algo, key in ((ordering.MIN_DEGREE, "mindeg"), (ordering.MIN_FILL, "minfill")):
            o, w = ordering.greedy_order(a, None, algo)
            assert o == c[key]["order"] and w == c[key]["widths"], (c["name"], key)


def brute_min_width(a):
    n = a.shape[0]
    best = n
    for perm in itertools.permutations(range(n)):
        best = min(best, max(ordering.replay_widths(a, perm)))
    return best


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_width_at_least_brute_force_minimum(seed):
    """No order beats the minimum over all orders (the treewidth, Sec. IV.B)."""
    rng = np.random.default_rng(seed)
    n = 7
    a = rng.random((n, n)) < 0.45
    a = np.triu(a, 1)
    a = a | a.T
    tw = brute_min_width(a)
    for algo in (ordering.MIN_FILL, ordering.MIN_DEGREE):
        _, w = ordering.greedy_order(a, None, algo)
        assert max(w) >= tw


def test_widths_of_known_graphs():
    """Trees have treewidth 1, cycles 2, K_n n-1; greedy reaches them."""
    tree = [(0, 1), (0, 2), (1, 3), (1, 4), (2, 5), (5, 6)]
    cyc = [(i, (i + 1) % 9) for i in range(9)]
    kn = list(itertools.combinations(range(6), 2))
    for edges, n, want in ((tree, 7, 1), (cyc, 9, 2), (kn, 6, 5)):
        for algo in (ordering.MIN_FILL, ordering.MIN_DEGREE):
            _, w = ordering.greedy_order(adj_of(n, edges), None, algo)
            assert max(w) == want


def test_replay_matches_greedy_profile():
    edges, g, b, z, t, nv, norm, adj = problem(30, 2, 5)
    o, w = ordering.greedy_order(adj)
    assert ordering.replay_widths(adj, o) == w


# ----------------------------- slicing ---------------------------------------

RULES = {"min-degree": ordering.MIN_DEGREE, "min-fill": ordering.MIN_FILL}


def test_slicing_hand_examples():
    """Step-dependent slicing worked by hand: min-degree and min-fill, r = 1 and r = 2,
    one and two rounds (rounds at s = 0 and s > 0, widths of earlier rounds counted)."""
    cases = load("slicing_hand.json")["cases"]
    assert {c["algo"] for c in cases} == set(RULES) and {c["r"] for c in cases} == {1, 2}
    for c in cases:
        a = adj_of(c["n"], c["edges"])
        plan = slicing.step_dependent_slicing(a, RULES[c["algo"]], c["width_limit"],
                                              c["max_vars"], c["r"])
        e = c["expect"]
        assert plan["sliced"] == e["sliced"], c["name"]
        assert plan["slice_step"] == e["slice_step"], c["name"]
        assert plan["order"] == e["order"], c["name"]
        assert plan["width"] == e["width"], c["name"]
        if "widths" in e:
            assert plan["widths"] == e["widths"], c["name"]
        if "rounds" in e:
            assert [[s, list(v)] for s, v in plan["rounds"]] == e["rounds"], c["name"]


def test_slicing_plan_widths_replay():
    """The plan's width profile is what eliminating its order on the graph gives
    (slice vertices removed at their round's step; later rounds' vertices still present
    during earlier segments)."""
    edges, g, b, z, t, nv, norm, adj = problem(24, 2, 8)
    plan = slicing.step_dependent_slicing(adj, ordering.MIN_FILL, 8, 4, 1)
    a = adj.copy()
    np.fill_diagonal(a, False)
    alive = np.ones(nv, dtype=bool)
    widths = []
    rounds = list(plan["rounds"])
    done = 0
    for i, v in enumerate(plan["order"]):
        while rounds and rounds[0][0] == i:
            for x in rounds.pop(0)[1]:
                ordering.remove_vertex(a, alive, x)
        nb = np.flatnonzero(a[v])
        widths.append(len(nb))
        ordering.eliminate(a, alive, v, nb)
        done += 1
    assert widths == plan["widths"]
    assert max(widths) == plan["width"]
    assert plan["width"] <= 8 or len(plan["sliced"]) == 4


# ----------------------------- ledger ----------------------------------------

def test_ledger_hand_example():
    """Path network A(x0) B(x0,x1) C(x1): step x0: m=2, u=2, c=1; step x1: m=2, u=1, c=0."""
    labels = [(0,), (0, 1), (1,)]
    tot, steps = ledger.ledger(labels, [0, 1])
    assert [(s["m"], s["u"], s["c"]) for s in steps] == [(2, 2, 1), (2, 1, 0)]
    # step 0: 6*(2-1)*4 + 2*(4-2) = 28 flops; bytes 8*(2+4+2) = 64
    # step 1: 6*(2-1)*2 + 2*(2-1) = 14 flops; bytes 8*(2+2+1) = 40
    assert [s["flops"] for s in steps] == [28, 14]
    assert [s["bytes"] for s in steps] == [64, 40]


def test_ledger_paper_numbers():
    pn = load("paper_numbers.json")
    # a rank-44 result in complex128
    b = ledger.step_bytes([], 44, elem_bytes=16)
    assert round(b / 1e12) == pn["width44_bytes_TB"]["value"]
    assert round(4 * 2 ** 44 / 1e12) == pn["width44_flops_T"]["value"]
    s = pn["slicing_speedup_64_nodes"]
    assert 2 ** (s["width_before"] - s["width_after"]) == s["value"]
    assert 2 ** pn["one_index_width_drop"]["value"] == pn["one_index_width_drop"]["speedup"]


def test_ledger_slicing_counts():
    """Per-slice steps drop sliced indices from every operand; prefix steps keep them."""
    edges, g, b, z, t, nv, norm, adj = problem(16, 2, 41)
    plan = slicing.step_dependent_slicing(adj, ordering.MIN_FILL, 5, 3, 1)
    tot, steps = ledger.ledger([l for l, _ in t], plan["order"], plan["sliced"], plan["slice_step"])
    k = len(plan["sliced"])
    assert tot["total_flops"] == tot["prefix_flops"] + tot["slice_flops"] * 2 ** k
    assert tot["slice_width"] <= plan["width"]
    assert all(s["c"] == s["u"] - 1 for s in steps)
    assert sum(1 for s in steps if s["region"] == "prefix") == tot["n_prefix_steps"]


# ----------------------------- energy ----------------------------------------

@pytest.mark.parametrize("n,p,seed", [(10, 1, 5), (12, 2, 6), (10, 3, 7)])
def test_lightcone_energy_equals_statevector(n, p, seed):
    edges, g, b, z = qaoa_instance(n, p, seed)
    e_sv = statevector.maxcut_energy(n, edges, g, b)
    e_lc, zz = energy.energy_lightcone(n, edges, p, g, b)
    assert abs(e_sv - e_lc) < 1e-11
    assert all(abs(x.imag if isinstance(x, complex) else 0.0) < 1e-12 for x in zz)


def test_p1_closed_form_energy_with_triangles():
    """Closed form with the triangle term, on graphs with triangles and mixed degrees."""
    graphs = [(4, list(itertools.combinations(range(4), 2))),
              (6, [(0, 1), (1, 2), (0, 2), (2, 3), (3, 4), (4, 5), (3, 5), (0, 5)])]
    for n, edges in graphs:
        for g, b in [(0.4, 0.3), (1.3, 2.1), (2.9, 0.7)]:
            zz = statevector.zz_expectations(n, edges, [g], [b])
            for (u, v), x in zip(edges, zz):
                cf = energy.edge_energy_p1_closed_form(n, edges, g, b, u, v)
                assert abs(cf - 0.5 * (1 - x)) < 1e-12


def test_p1_closed_form_on_3_regular():
    n = 12
    edges, g, b, z = qaoa_instance(n, 1, 9)
    e = sum(energy.edge_energy_p1_closed_form(n, edges, g[0], b[0], u, v) for u, v in edges)
    assert abs(e - statevector.maxcut_energy(n, edges, g, b)) < 1e-11


# ----------------------------- proposal MLP ----------------------------------

def _mlp_case(nf=5, hidden=7, batch=9, seed=4):
    from oracle import mlp
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.6, mlp.n_params(nf, hidden))
    x = rng.normal(0, 1, (batch, nf))
    t = rng.normal(0, 1, batch)
    return p, x, t


def test_mlp_gradients_match_finite_differences():
    """The oracle's chain-rule gradients against central differences of its loss (FP64)."""
    from oracle import mlp
    nf, hidden = 5, 7
    p, x, t = _mlp_case(nf, hidden)
    g = mlp.gradients(p, x, t, nf, hidden)
    h = 1e-6
    fd = np.zeros_like(p)
    for i in range(len(p)):
        e = np.zeros_like(p)
        e[i] = h
        fd[i] = (mlp.loss(p + e, x, t, nf, hidden) - mlp.loss(p - e, x, t, nf, hidden)) / (2 * h)
    assert np.max(np.abs(fd - g)) <= 1e-7 * max(1.0, np.max(np.abs(g)))


def test_adam_first_step_is_signed_lr():
    """Adam's first step (bias-corrected m = g, v = g^2) moves each parameter by lr*sign(g)."""
    from oracle import mlp
    p = np.array([0.5, -1.0, 2.0])
    g = np.array([0.3, -2.0, 1e-3])
    p1, m, v = mlp.adam_step(p, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    assert np.allclose(p1, p - 0.01 * np.sign(g), atol=1e-7)


def test_proposal_candidate_counts():
    """One candidate per (step up to the first peak, top-degree vertex); labels never exceed 1
    by more than the prefix allows and the paper's max-degree candidate is rank 0."""
    from oracle import proposal
    edges, g, b, z, t, nv, norm, adj = problem(20, 2, 3)
    order, widths = ordering.greedy_order(adj)
    peak = int(np.argmax(widths))
    cands = proposal.round_candidates(adj, order, widths, nv, 3)
    assert len(cands) == 3 * (peak + 1)
    assert all(c[2] == i % 3 for i, c in enumerate(cands))
    F, L, M = proposal.dataset(adj, ordering.MIN_FILL, 3)
    assert F.shape == (3 * (peak + 1), 16) and np.all(L > 0) and np.all(L <= 1.0 + 1e-12)


# ------------------------ launch groups (fusion rule) -------------------------

def test_launch_groups_hand_examples():
    """The fusion rule's grouping worked by hand: joins, and launches cut by union
    containment, by max_nsum, by max_ops, by a bucket without the previous result, and
    by the slice boundary (sliced indices dropped from per-slice tensors)."""
    for c in load("launch_groups_hand.json")["cases"]:
        got = ledger.launch_groups(c["tensors"], c["order"], c["sliced"], c["slice_step"],
                                   max_nsum=c["max_nsum"], max_ops=c["max_ops"])
        assert got == c["expect"], c["name"]


# ----------------------------- proposal features -------------------------------

def _feature_value(f):
    if isinstance(f, str):  # "log2(k)/d"
        num, den = f.split("/")
        return math.log2(float(num[len("log2("):-1])) / float(den)
    return f[0] / f[1]


def test_proposal_features_hand_example():
    """Every one of the 16 features of four candidates, and their labels, worked by hand
    on a five-vertex graph."""
    from oracle import proposal
    g = load("proposal_hand.json")
    a = adj_of(g["n"], g["edges"])
    order, widths = ordering.greedy_order(a, None, ordering.MIN_DEGREE)
    assert order == g["order"] and widths == g["widths"]
    base = proposal.round_candidates(a, order, widths, g["n"], g["topv"])
    assert len(base) == g["n_candidates"]
    for c in g["candidates"]:
        cands = base if "topv" not in c else proposal.round_candidates(a, order, widths, g["n"],
                                                                       c["topv"])
        hit = [f for s, v, j, f in cands if (s, v, j) == (c["s"], c["v"], c["j"])]
        assert len(hit) == 1, c
        want = [_feature_value(x) for x in c["features"]]
        assert len(want) == 16
        assert np.allclose(hit[0], want, rtol=0, atol=1e-12), (c["s"], c["v"], hit[0], want)
        w = proposal.candidate_width(a, order, widths, c["s"], c["v"], ordering.MIN_DEGREE)
        assert w == c["label_width"], (c["s"], c["v"], w)


# ------------------------------ MLP forward ------------------------------------

def test_mlp_forward_hand_example():
    """Forward values, loss and two gradients of the proposal MLP worked by hand."""
    from oracle import mlp
    g = load("mlp_hand.json")
    params = np.concatenate([np.ravel(g["W1"]), g["b1"], np.ravel(g["W2"]), g["b2"], g["w3"],
                             [g["b3"]]])
    assert len(params) == mlp.n_params(g["nf"], g["hidden"])
    y, _ = mlp.forward(params, g["x"], g["nf"], g["hidden"])
    assert np.array_equal(y, np.array(g["y"]))  # exact in binary floating point
    L = mlp.loss(params, g["x"], g["t"], g["nf"], g["hidden"])
    assert abs(L - g["loss"][0] / g["loss"][1]) <= 1e-15
    grad = mlp.gradients(params, g["x"], g["t"], g["nf"], g["hidden"])
    assert abs(grad[-1] - g["grad_b3"]) <= 1e-15
    gw3 = [_feature_value(x) if isinstance(x, list) else x for x in g["grad_w3"]]
    assert np.allclose(grad[-1 - g["hidden"]:-1], gw3, rtol=0, atol=1e-15)


def test_step_proposal_hand_example():
    """Candidates, all 16 features and the rollout labels of two elimination-step
    candidates, worked by hand on a five-vertex graph."""
    from oracle import proposal
    g = load("step_proposal_hand.json")
    a = adj_of(g["n"], g["edges"])
    feats, labels, meta = proposal.order_dataset(a, ordering.MIN_FILL, g["topc"], g["stride"])
    at0 = [m[1] for m in meta if m[0] == 0]
    assert at0 == g["candidates"]
    for v, want in g["features"].items():
        i = [q for q, m in enumerate(meta) if m[0] == 0 and m[1] == int(v)][0]
        assert np.allclose(feats[i], [_feature_value(x) for x in want], rtol=0, atol=1e-12), v
        assert abs(labels[i] - math.log2(g["labels_log2_of"][v])) <= 1e-12
