"""Seeded random streams for the synthetic workloads.

Input generation only: nothing here computes any step of the receive path.

Two generators are used:

* ``SplitMix64`` -- Steele, Lea and Flood's 64-bit mixer ("Fast splittable
  pseudorandom number generators", OOPSLA 2014), written out in pure Python
  integers so that its output is identical on every machine.  It draws the
  base matrices (whose bytes are frozen by a SHA-256 in the tests) and splits a
  config seed into independent sub-stream seeds.
* NumPy ``Generator(PCG64(seed))`` seeded from a SplitMix64 draw, for bulk
  draws (payload bits, noise, puncture masks).  Those are regenerated in the
  same process that checks them, so they need no cross-machine freeze.
"""
from __future__ import annotations

import numpy as np

_M64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64: state += golden gamma, then two xor-shift-multiply rounds."""

    def __init__(self, seed: int):
        self.state = seed & _M64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def below(self, n: int) -> int:
        """Uniform integer in [0, n) by rejection (no modulo bias)."""
        if n <= 0:
            raise ValueError("n must be positive")
        limit = ((1 << 64) // n) * n
        while True:
            x = self.next_u64()
            if x < limit:
                return x % n

    def bernoulli(self, p: float) -> bool:
        return self.uniform() < p

    def sample_distinct(self, population: list, k: int) -> list:
        """k distinct items of ``population`` by a partial Fisher-Yates shuffle."""
        pool = list(population)
        for i in range(k):
            j = i + self.below(len(pool) - i)
            pool[i], pool[j] = pool[j], pool[i]
        return pool[:k]


def derive_seed(*path: int) -> int:
    """A 64-bit seed for the sub-stream named by an integer path.

    ``derive_seed(cfg_seed, purpose, index)`` mixes each element in turn, so
    sub-streams for different (slot, UE, CB) indices are independent.
    """
    s = SplitMix64(0x243F6A8885A308D3)
    acc = s.next_u64()
    for p in path:
        s = SplitMix64(acc ^ (p & _M64))
        acc = s.next_u64()
    return acc


def np_stream(*path: int) -> np.random.Generator:
    """A NumPy PCG64 generator seeded from ``derive_seed(*path)``."""
    return np.random.Generator(np.random.PCG64(derive_seed(*path)))
