"""Oracle: the QAOA MaxCut amplitude as a binary-index tensor network (FP64).

TEST INFRASTRUCTURE. This package is the plain, slow CPU oracle that the CUDA
path is checked against. Only tests, the smoke check and the benchmark's CPU
baseline leg may import it; the product path never does.

Tensor expression (Sec. IV.A, Table I) in the line-graph form with diagonal
gates (Sec. IV.B, Fig. 2): a vertex is a binary index, a tensor is a clique on
its indices, a diagonal two-qubit gate keeps only the two input indices.

Readings taken where the paper is silent or garbled (Sec. III.A):
  * C = sum over edges (u, v) of (1 - Z_u Z_v) / 2, so exp(-i gamma C) gives the
    basis state x the phase exp(-i gamma cut(x));
  * the layers use gamma_k, beta_k (k = 1..p), layer 1 acting first;
  * |psi_0> = |+>^N; the amplitude returned is <z|psi_p>.

Variables: (v, k) for qubit v and time k = 0..p-1 with id k*N + v.
Tensors, in this order:
  1. for each v: |+> = (1, 1) on (v, 0) (normalisation 2^(-N/2) kept aside);
  2. for k = 1..p: for each edge (u, v) in edge order the diagonal phase
     D(a, b) = exp(-i gamma_k [a != b]) on ((u, k-1), (v, k-1)); then for each v
     the mixer M(a, a') = <a'| exp(-i beta_k X) |a> on ((v, k-1), (v, k)) when
     k < p, or, when k = p, the row a' = z_v of it as a vector on (v, p-1).
"""

from __future__ import annotations

import math

import numpy as np


def var_id(v: int, k: int, n: int) -> int:
    return k * n + v


def mixer_matrix(beta: float) -> np.ndarray:
    """M[a, a'] = <a'| exp(-i beta X) |a> = cos(beta) if a == a' else -i sin(beta)."""
    c, s = math.cos(beta), math.sin(beta)
    return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)


def phase_matrix(gamma: float) -> np.ndarray:
    """D[a, b] = exp(-i gamma [a != b]): one edge term of exp(-i gamma C)."""
    e = complex(math.cos(gamma), -math.sin(gamma))
    return np.array([[1.0, e], [e, 1.0]], dtype=np.complex128)


def build_network(n, edges, p, gammas, betas, z, open_qubits=()):
    """Tensors of <z| U(gamma, beta) |+>^N, unnormalised.

    Returns (tensors, n_vars, norm): tensors is a list of (labels, data) with
    labels a tuple of variable ids and data an ndarray of shape (2,)*len(labels)
    whose axis t is labels[t]; the amplitude is norm * (full contraction).

    Several amplitudes (Sec. VII): for the j-th qubit v of open_qubits the last
    mixer keeps its output index as the variable n*p + j instead of being folded
    with z_v; the contraction is then a tensor over those a variables whose entry
    b (bit j = b_j) is the amplitude of z with z_v replaced by b_j.
    """
    if p < 1:
        raise ValueError("p must be >= 1")
    if len(gammas) != p or len(betas) != p or len(z) != n:
        raise ValueError("length mismatch")
    open_index = {v: j for j, v in enumerate(open_qubits)}
    if len(open_index) != len(open_qubits) or any(not 0 <= v < n for v in open_qubits):
        raise ValueError("bad open qubits")
    tensors = []
    plus = np.array([1.0, 1.0], dtype=np.complex128)
    for v in range(n):
        tensors.append(((var_id(v, 0, n),), plus.copy()))
    for k in range(1, p + 1):
        dmat = phase_matrix(gammas[k - 1])
        mmat = mixer_matrix(betas[k - 1])
        for (u, v) in edges:
            tensors.append(((var_id(u, k - 1, n), var_id(v, k - 1, n)), dmat.copy()))
        for v in range(n):
            if k < p:
                tensors.append(((var_id(v, k - 1, n), var_id(v, k, n)), mmat.copy()))
            elif v in open_index:
                tensors.append(((var_id(v, p - 1, n), n * p + open_index[v]), mmat.copy()))
            else:
                tensors.append(((var_id(v, p - 1, n),), mmat[:, z[v]].copy()))
    return tensors, n * p + len(open_index), 2.0 ** (-n / 2.0)


def open_clique(adj_sets, n, p, a):
    """The clique the open variables form (Sec. VII: the result tensor over them)."""
    opens = [n * p + j for j in range(a)]
    for x in opens:
        for y in opens:
            if x != y:
                adj_sets[x].add(y)
    return adj_sets


def line_graph(tensors, n_vars):
    """Adjacency sets of the line graph: vertices are indices, each tensor a clique."""
    adj = [set() for _ in range(n_vars)]
    for labels, _ in tensors:
        for a in labels:
            for b in labels:
                if a != b:
                    adj[a].add(b)
    return adj
