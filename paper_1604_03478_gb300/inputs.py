"""Seeded synthetic inputs shared by the tests and the benchmark.

This module draws random numbers only; it holds none of the method's
arithmetic (lattice weights, equilibria and the like are passed in by the
caller).
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def gaussian_field(shape, sigma: float, seed: int) -> np.ndarray:
    """i.i.d. N(0, sigma^2) per entry (e.g. a hot-wall perturbation field)."""
    return rng(seed).normal(0.0, sigma, size=shape)


def noisy(base: np.ndarray, rel: float, seed: int) -> np.ndarray:
    """base * (1 + rel * U(-1, 1)) elementwise."""
    return base * (1.0 + rel * rng(seed).uniform(-1.0, 1.0, size=base.shape))


def uniform(shape, lo: float, hi: float, seed: int) -> np.ndarray:
    return rng(seed).uniform(lo, hi, size=shape)


def ensemble(n: int, seed: int, sizes=(48, 64, 96, 128, 160), log_ra=(4.0, 6.0), ste=(0.05, 0.2),
             faces=(0, 1)):
    """Parameter draws of an ensemble of cavities: edge length uniform over
    ``sizes``, Ra log-uniform, Ste uniform, heated face uniform."""
    r = rng(seed)
    out = []
    for _ in range(n):
        out.append(dict(n=int(r.choice(sizes)), Ra=float(10 ** r.uniform(*log_ra)),
                        Ste=float(r.uniform(*ste)), face=int(r.choice(faces))))
    return out
