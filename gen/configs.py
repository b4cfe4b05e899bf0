"""Recipes of the five benchmark workloads: sizes, densities, seeds and planted
squares of every matrix.  Input drawing only (the cells come from the seeded
generator of this package); none of the maximal-square arithmetic.

Each matrix is a dict ``{m, n, p, seed, plant}``: an m x n Bernoulli(p)
matrix of the generator's stream ``seed``, plus an all-ones plant x plant
square at ``plant_pos(seed, m, n, plant)`` when ``plant > 0``.

  c1  256 x 256, p = 0.5, seed 0 (with the int32 dp map)
  c2  square sides 1000..5000 x densities 0.1..0.9, seed 10*side/1000 + 10p
      (the paper's size x density grid, Sec. 4.1 and Sec. 4.6)
  c3  32768 x 32768, p = 0.9, one planted 600-square, seed 3
  c4  4096 matrices, m and n log-uniform in [16, 2048], density uniform over
      0.1..0.9, half with a planted square of side uniform in [1, min(m, n)]
  c5  serving stream: square sides log-uniform in [64, 8192], density uniform
      in [0.1, 0.9], one seeded matrix per request (bit-packed on the wire)
"""
from __future__ import annotations

import math

from . import draw


def c1_spec() -> dict:
    return dict(m=256, n=256, p=0.5, seed=0, plant=0)


def c2_specs() -> list[dict]:
    specs = []
    for side in (1000, 2000, 3000, 4000, 5000):
        for k in range(1, 10):
            specs.append(dict(m=side, n=side, p=k / 10, seed=10 * (side // 1000) + k, plant=0))
    return specs


def c3_spec() -> dict:
    return dict(m=32768, n=32768, p=0.9, seed=3, plant=600)


def _unit(seed: int, j: int) -> float:
    """Uniform [0, 1) from draw j of a matrix's parameter stream (53 bits)."""
    return (draw(seed, (1 << 40) + j) >> 11) / float(1 << 53)


def c4_specs(count: int = 4096) -> list[dict]:
    lo, hi = math.log(16), math.log(2049)
    specs = []
    for k in range(count):
        seed = draw(4, k)
        m = min(2048, int(math.exp(lo + (hi - lo) * _unit(seed, 0))))
        n = min(2048, int(math.exp(lo + (hi - lo) * _unit(seed, 1))))
        p = (1 + int(9 * _unit(seed, 2))) / 10
        plant = 1 + int(min(m, n) * _unit(seed, 4)) if _unit(seed, 3) < 0.5 else 0
        specs.append(dict(m=m, n=n, p=p, seed=seed, plant=plant))
    return specs


def c5_specs(count: int = 20000) -> list[dict]:
    """Request k: side log-uniform in [64, 8192], density uniform in [0.1, 0.9]
    (continuous, no quantisation), its own stream draw(5, k)."""
    lo, hi = math.log(64), math.log(8193)
    specs = []
    for k in range(count):
        seed = draw(5, k)
        side = min(8192, int(math.exp(lo + (hi - lo) * _unit(seed, 0))))
        p = 0.1 + 0.8 * _unit(seed, 1)
        specs.append(dict(m=side, n=side, p=p, seed=seed, plant=0))
    return specs
