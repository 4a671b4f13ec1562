"""Oracle: brute-force 2^N statevector of the QAOA ansatz (Sec. III.A), N <= 20.

TEST INFRASTRUCTURE (see oracle/network.py).

|psi_p> = prod_k exp(-i beta_k B) exp(-i gamma_k C) |+>^N with B = sum_v X_v and
C = sum_E (1 - Z_u Z_v)/2, layer 1 first. Basis state x carries bit v of qubit
v. The cost layer multiplies x by exp(-i gamma cut(x)); the mixer layer is one
2x2 rotation cos(beta) I - i sin(beta) X per qubit.
"""

from __future__ import annotations

import math

import numpy as np


def cut_values(n, edges):
    x = np.arange(1 << n, dtype=np.int64)
    cut = np.zeros(1 << n, dtype=np.int64)
    for (u, v) in edges:
        cut += ((x >> u) ^ (x >> v)) & 1
    return cut


def qaoa_state(n, edges, gammas, betas):
    if n > 22:
        raise ValueError("statevector limited to small n")
    psi = np.full(1 << n, 2.0 ** (-n / 2.0), dtype=np.complex128)
    cut = cut_values(n, edges)
    for g, b in zip(gammas, betas):
        psi *= np.exp(-1j * g * cut)
        c, s = math.cos(b), math.sin(b)
        for q in range(n):
            t = psi.reshape(-1, 2, 1 << q)
            a0 = t[:, 0, :].copy()
            a1 = t[:, 1, :].copy()
            t[:, 0, :] = c * a0 - 1j * s * a1
            t[:, 1, :] = -1j * s * a0 + c * a1
    return psi


def amplitude(n, edges, gammas, betas, z):
    psi = qaoa_state(n, edges, gammas, betas)
    idx = sum(int(b) << v for v, b in enumerate(z))
    return complex(psi[idx])


def zz_expectations(n, edges, gammas, betas):
    """<Z_u Z_v> for every edge, from |psi|^2."""
    prob = np.abs(qaoa_state(n, edges, gammas, betas)) ** 2
    x = np.arange(1 << n, dtype=np.int64)
    out = []
    for (u, v) in edges:
        sign = 1 - 2 * (((x >> u) ^ (x >> v)) & 1)
        out.append(float(np.dot(prob, sign)))
    return out


def maxcut_energy(n, edges, gammas, betas):
    """<C> = sum over edges of (1 - <Z_u Z_v>) / 2."""
    return sum(0.5 * (1.0 - zz) for zz in zz_expectations(n, edges, gammas, betas))
