"""Seeded synthetic generator matrices for the five workloads.

This module holds no arithmetic of the method: it only draws random
generator matrices ``G = [I_k | A]`` over F_p with numpy's PCG64 generator,
so that the CUDA path, the CPU oracle, the tests and the benchmark all see
identical bytes.  The paper's own matrices (its Magma/Guava datasets, Sec. 5)
are not published; random systematic codes of the same shape stand in for
them (Sec. 5.2.1 and Sec. 5.3 describe random matrices with k <= 25, n <= 58
over F_7 and k <= 50, n <= 74 over F_3).
"""
from __future__ import annotations

import hashlib
import math
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Code:
    """One linear code: prime ``p``, length ``n``, dimension ``k`` and a
    ``k x n`` uint8 generator matrix with entries in ``[0, p)``."""

    p: int
    n: int
    k: int
    G: np.ndarray

    def digest(self) -> str:
        h = hashlib.sha256()
        h.update(np.array([self.p, self.n, self.k], dtype=np.int64).tobytes())
        h.update(np.ascontiguousarray(self.G, dtype=np.uint8).tobytes())
        return h.hexdigest()


def systematic(p: int, n: int, k: int, A: np.ndarray) -> Code:
    """``G = [I_k | A]`` as uint8."""
    G = np.hstack([np.eye(k, dtype=np.uint8), np.asarray(A, dtype=np.uint8)])
    return Code(int(p), int(n), int(k), np.ascontiguousarray(G))


def single_code(seed: int, p: int, n: int, k: int) -> Code:
    """Random ``[n, k]`` code over F_p: ``A`` uniform in ``[0, p)`` from PCG64(seed)."""
    rng = np.random.default_rng(seed)
    A = rng.integers(0, p, size=(k, n - k), dtype=np.uint8)
    return systematic(p, n, k, A)


# The three single-code workloads: (seed, p, n, k).
SINGLE = {
    "f3_n30_k15": (0, 3, 30, 15),
    "f7_n40_k20": (1, 7, 40, 20),
    "f3_n80_k40": (2, 3, 80, 40),
}


def single(name: str) -> Code:
    return single_code(*SINGLE[name])


def batch_codes(count: int = 512, seed: int = 3) -> list[Code]:
    """Batched workload: per code p in {3,7}, n in {24,28,...,64},
    k = round(r n) with r uniform in [1/3, 2/3], A uniform in F_p."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        p = int(rng.choice([3, 7]))
        n = int(rng.choice(np.arange(24, 65, 4)))
        r = float(rng.uniform(1.0 / 3.0, 2.0 / 3.0))
        k = int(round(r * n))
        A = rng.integers(0, p, size=(k, n - k), dtype=np.uint8)
        out.append(systematic(p, n, k, A))
    return out


def serve_codes(count: int = 10000, seed: int = 4, rate: float = 200.0):
    """Serving workload: per code p in {3,5,7}, n uniform in [20,72],
    k uniform in [ceil(n/3), floor(2n/3)], A uniform in F_p; then Poisson
    inter-arrival gaps with mean 1/rate seconds, drawn after all codes.
    Returns ``(codes, arrival_times_seconds)``."""
    rng = np.random.default_rng(seed)
    codes = []
    for _ in range(count):
        p = int(rng.choice([3, 5, 7]))
        n = int(rng.integers(20, 73))
        k = int(rng.integers(math.ceil(n / 3), (2 * n) // 3 + 1))
        A = rng.integers(0, p, size=(k, n - k), dtype=np.uint8)
        codes.append(systematic(p, n, k, A))
    gaps = rng.exponential(1.0 / rate, size=count)
    return codes, np.cumsum(gaps)


def random_code(rng: np.random.Generator, p: int, n: int, k: int, systematic_form: bool = False) -> Code:
    """A random k x n matrix over F_p (not necessarily full rank unless
    ``systematic_form``), for property tests."""
    if systematic_form:
        A = rng.integers(0, p, size=(k, n - k), dtype=np.uint8)
        return systematic(p, n, k, A)
    G = rng.integers(0, p, size=(k, n), dtype=np.uint8)
    return Code(p, n, k, G)
