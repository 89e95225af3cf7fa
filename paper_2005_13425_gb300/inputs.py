"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module only draws random numbers and sizes; it holds none of the
method's arithmetic (no GLL points, derivative matrix, geometry, operator,
numbering or solver).  Both the CUDA path and the oracle receive exactly the
arrays produced here.

Workload recipe (the paper's workload is Nekbone's own synthetic box mesh,
arXiv 2005.13425 Sec. III and V: a cubic domain of hexahedral elements,
E = 64..4096 elements, polynomial degree 9 for the headline runs):

* the mesh perturbation coefficients s_d, d = x, y, z, are uniform in [-1, 1];
* a right-hand side is uniform in [-1, 1] per unique global node (so it is
  continuous across elements) and is copied to every local copy by each side
  with its own numbering;
* an operator input u is uniform in [-1, 1] per local point.
"""
from __future__ import annotations

import math

import numpy as np

# Seeds of the standard configurations.
SEED_MESH = 0     # perturbation coefficients
SEED_F = 1        # right-hand side per unique node
SEED_U = 2        # operator input per local point
PERTURB_AMP = 0.05


def perturbation_coeffs(seed: int = SEED_MESH) -> np.ndarray:
    """s_d uniform in [-1, 1] for the sinusoidal mesh perturbation."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=3)


def unique_grid_shape(Ex: int, Ey: int, Ez: int, n: int):
    """Number of unique GLL nodes per direction of an Ex x Ey x Ez box."""
    return (Ex * (n - 1) + 1, Ey * (n - 1) + 1, Ez * (n - 1) + 1)


def unique_field(Ex: int, Ey: int, Ez: int, n: int, seed: int = SEED_F) -> np.ndarray:
    """Uniform [-1, 1] values, one per unique node, x fastest."""
    NX, NY, NZ = unique_grid_shape(Ex, Ey, Ez, n)
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=NX * NY * NZ)


def local_field(E: int, n: int, seed: int = SEED_U) -> np.ndarray:
    """Uniform [-1, 1] values per local point, shape [E, n^3]."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=(E, n ** 3))


def box_dims(E: int):
    """Box dimensions for a requested element count: k = round(log2 E),
    dims 2^a x 2^b x 2^c with a >= b >= c, a - c <= 1, a + b + c = k."""
    k = max(0, int(round(math.log2(max(1, E)))))
    c = k // 3
    rem = k - 3 * c
    a = c + (1 if rem >= 1 else 0)
    b = c + (1 if rem >= 2 else 0)
    return (1 << a, 1 << b, 1 << c)


def batch_problems(count: int, seed: int, e_lo: int = 64, e_hi: int = 4096,
                   degrees=(6, 8, 10, 12)):
    """Problem list for batched / served solves: E log-uniform in
    [e_lo, e_hi] rounded to box dims, n drawn from ``degrees`` (GLL points
    per direction), per-problem perturbation seed."""
    rng = np.random.default_rng(seed)
    out = []
    for pid in range(count):
        E = float(np.exp(rng.uniform(math.log(e_lo), math.log(e_hi))))
        dims = box_dims(int(round(E)))
        n = int(rng.choice(degrees))
        out.append(dict(id=pid, dims=dims, n=n, mesh_seed=seed * 100003 + pid,
                        f_seed=seed * 100003 + pid + 7919))
    return out
