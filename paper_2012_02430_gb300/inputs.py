"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the simulation method itself: it only draws
problem instances. The paper's workload is MaxCut QAOA on random 3-regular
graphs (Sec. III.B), with angles and a target bitstring; every draw below comes
from one counter-based generator, SplitMix64 (Steele, Lea, Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014), so that a seed fixes
an instance on every machine.
"""

from __future__ import annotations

import math

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64: a 64-bit Weyl sequence passed through a fixed mixing function."""

    GOLDEN = 0x9E3779B97F4A7C15

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + self.GOLDEN) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def below(self, n: int) -> int:
        """Integer in [0, n) for n < 2**32 (multiply-shift of the top 32 bits)."""
        if not 0 < n < (1 << 32):
            raise ValueError("n out of range")
        return ((self.next_u64() >> 32) * n) >> 32

    def uniform(self) -> float:
        """Double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))


def random_regular_graph(n: int, d: int, seed: int, max_tries: int = 100000):
    """Simple random d-regular graph on n vertices by the pairing (configuration) model.

    n*d stubs are shuffled with Fisher-Yates and paired consecutively; a pairing
    with a self-loop or a repeated edge is rejected and drawn again. Returns the
    edge list sorted lexicographically, each edge as (u, v) with u < v.
    """
    if n * d % 2 or d >= n or n <= 0 or d < 0:
        raise ValueError("no simple d-regular graph with these n, d")
    rng = SplitMix64(seed)
    for _ in range(max_tries):
        stubs = [v for v in range(n) for _ in range(d)]
        for i in range(len(stubs) - 1, 0, -1):
            j = rng.below(i + 1)
            stubs[i], stubs[j] = stubs[j], stubs[i]
        edges = set()
        ok = True
        for i in range(0, len(stubs), 2):
            u, v = stubs[i], stubs[i + 1]
            if u == v:
                ok = False
                break
            e = (min(u, v), max(u, v))
            if e in edges:
                ok = False
                break
            edges.add(e)
        if ok:
            return sorted(edges)
    raise RuntimeError("pairing model did not produce a simple graph")


def random_angles(p: int, seed: int):
    """gamma_k, beta_k uniform in [0, pi) for k = 1..p (two lists of length p)."""
    rng = SplitMix64(seed ^ 0xA5A5A5A5A5A5A5A5)
    gammas = [math.pi * rng.uniform() for _ in range(p)]
    betas = [math.pi * rng.uniform() for _ in range(p)]
    return gammas, betas


def random_bitstring(n: int, seed: int):
    """n uniform bits (list of 0/1)."""
    rng = SplitMix64(seed ^ 0x5A5A5A5A5A5A5A5A)
    return [int(rng.next_u64() >> 63) for _ in range(n)]


def qaoa_instance(n: int, p: int, seed: int, d: int = 3):
    """One seeded QAOA MaxCut instance: (edges, gammas, betas, bitstring)."""
    edges = random_regular_graph(n, d, seed)
    gammas, betas = random_angles(p, seed)
    z = random_bitstring(n, seed)
    return edges, gammas, betas, z


def random_slice_ids(k: int, count: int, seed: int):
    """count slice ids uniform in [0, 2^k) (k <= 64), from SplitMix64."""
    rng = SplitMix64(seed ^ 0x3C3C3C3C3C3C3C3C)
    mask = (1 << k) - 1
    return [rng.next_u64() & mask for _ in range(count)]
