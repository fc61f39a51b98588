"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests and
the benchmark.

This module holds none of the lattice Boltzmann arithmetic: it only draws porosity
fields and workload descriptions.  Random numbers the method itself draws (the
start-temperature noise) are not made here; both implementations generate those
from the SplitMix64 definition.

Porosity recipe (the paper's problems use uniform porosity; the variable fields are
synthetic stand-ins shaped like REV-scale packed beds, Eq. 8 and ref. [43]):
white noise uniform in [lo, hi] from numpy's PCG64 seeded with `seed`, smoothed by
a Gaussian of standard deviation `sigma` cells, truncated at 4 sigma, reflected at
the edges.
"""
from __future__ import annotations

import math

import numpy as np


def porosity_field(nr: int, nz: int, lo: float, hi: float, sigma: float, seed: int) -> np.ndarray:
    """float32 (nr, nz) porosity, z fastest."""
    rng = np.random.Generator(np.random.PCG64(seed))
    white = rng.uniform(lo, hi, size=(nr, nz))
    if sigma > 0:
        from scipy.ndimage import gaussian_filter

        white = gaussian_filter(white, sigma=sigma, mode="reflect", truncate=4.0)
    return np.ascontiguousarray(white, dtype=np.float32)


def porosity_field_around(nr: int, nz: int, mean: float, amp: float, sigma: float, seed: int) -> np.ndarray:
    """Smoothed porosity field with a prescribed mean and standard deviation: white
    noise smoothed by a Gaussian of sigma cells (as porosity_field), standardised,
    scaled to standard deviation `amp` around `mean`, clipped to [0.05, 0.99]."""
    s = porosity_field(nr, nz, 0.0, 1.0, sigma, seed).astype(np.float64)
    s = (s - s.mean()) / max(s.std(), 1e-12)
    return np.ascontiguousarray(np.clip(mean + amp * s, 0.05, 0.99), dtype=np.float32)


def uniform_field(nr: int, nz: int, value: float) -> np.ndarray:
    return np.full((nr, nz), value, dtype=np.float32)


def sweep_instances(n: int, seed: int, nr_lo: int = 64, nr_hi: int = 512):
    """Parameter draws of the batched sweep: Nr ~ U{nr_lo..nr_hi}, Nz = 2 Nr,
    Ra log-uniform [1e3, 1e6], Da log-uniform [1e-5, 1e-1], eps ~ U[0.3, 0.9],
    Pr in {0.71, 1, 7}, R* ~ U[1.5, 4]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n):
        nr = int(rng.integers(nr_lo, nr_hi + 1))
        out.append(dict(
            nr=nr, nz=2 * nr,
            Ra=float(10 ** rng.uniform(3, 6)),
            Da=float(10 ** rng.uniform(-5, -1)),
            eps=float(rng.uniform(0.3, 0.9)),
            Pr=float(rng.choice([0.71, 1.0, 7.0])),
            radius_ratio=float(rng.uniform(1.5, 4.0)),
        ))
    return out


def subsample_shape(nr: int, nz: int, factor: int):
    return int(math.ceil(nr / factor)), int(math.ceil(nz / factor))
