"""Seeded synthetic inputs shared by the oracle-side and the GPU-side tests.

Only random numbers live here (no arithmetic of the method): fields are drawn
from numpy's default_rng with a fixed seed, in the library's layout sizes.
"""
import numpy as np


def rng(seed=0):
    return np.random.default_rng(seed)


def field(n, seed=0, scale=1.0):
    return scale * rng(seed).standard_normal(n)


def positive_field(n, seed=0, lo=0.5, hi=1.5):
    return lo + (hi - lo) * rng(seed).random(n)
