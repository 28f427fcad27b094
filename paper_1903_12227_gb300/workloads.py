"""Seeded synthetic workloads: realization descriptors only.

This module holds no arithmetic of the method.  It lists, for each benchmark
configuration, the realization descriptors (cell count L per axis, grid cells
per unit length m0, inclusion side in grid cells, inclusion count, the two
coefficient values, run seed and realization index).  The random inclusion
corners themselves are drawn inside the method (``gen_field``) from
(seed, index), by each implementation from the published SplitMix64
definition.

Where a configuration mixes sizes or contrasts (the uneven batch), the per
realization L and contrast are workload inputs drawn here with numpy's
seeded generator.

Configurations (all synthetic; the paper uses no dataset):

* ``single_L4``   -- L=4, h=1/8 (32x32 nodes), 11 inclusions of side 1,
  contrast 10, tol 1e-12, one realization.
* ``plain_L32``   -- L=32, h=1/16 (512x512 nodes), 717 inclusions of side 1,
  contrast 10, tol 1e-10, 1000 realizations.
* ``uneven_4096`` -- 4096 realizations, L uniform in {8,16,32,64}, h=1/8,
  contrast uniform in {10,100}.
* ``adjoint_L64`` -- L=64, h=1/16 (1024x1024 nodes), 2867 inclusions,
  contrast 100, batch 64.
* ``large_L256``  -- L=256, h=1/8 (2048x2048 nodes), 45875 inclusions,
  contrast 100, 256 realizations.

Inclusion count = round(0.7 L^2) (density 0.7 per unit area), inclusion side
= one unit length = m0 grid cells.  The 3D realizations (``realization3``)
place round(0.7 L^3) unit cubes on [0,L)^3.
"""
from __future__ import annotations

import numpy as np

DENSITY = 0.7


def realization(L: int, m0: int, contrast: float, seed: int, index: int,
                density: float = DENSITY, side_units: float = 1.0,
                a_matrix: float = 1.0) -> dict:
    """Descriptor of one realization (inclusion side side_units, in unit lengths)."""
    s = int(round(side_units * m0))
    return {"L": int(L), "m0": int(m0), "incl_cells": s,
            "n_incl": int(round(density * L * L)),
            "a_matrix": float(a_matrix), "a_incl": float(contrast) * float(a_matrix),
            "seed": int(seed), "index": int(index)}


def realization3(L: int, m0: int, contrast: float, seed: int, index: int,
                 density: float = DENSITY, side_units: float = 1.0,
                 a_matrix: float = 1.0) -> dict:
    """Descriptor of one 3D realization on [0,L)^3: round(density L^3) cubes
    of side side_units (the 2D recipe with areas replaced by volumes)."""
    s = int(round(side_units * m0))
    return {"L": int(L), "m0": int(m0), "incl_cells": s,
            "n_incl": int(round(density * L * L * L)),
            "a_matrix": float(a_matrix), "a_incl": float(contrast) * float(a_matrix),
            "seed": int(seed), "index": int(index)}


def batch(L: int, m0: int, contrast: float, seed: int, count: int, start: int = 0,
          **kw) -> list:
    return [realization(L, m0, contrast, seed, start + k, **kw) for k in range(count)]


CONFIGS = {
    "single_L4": dict(L=4, m0=8, contrast=10.0, count=1, tol=1e-12),
    "plain_L32": dict(L=32, m0=16, contrast=10.0, count=1000, tol=1e-10),
    "uneven_4096": dict(Ls=(8, 16, 32, 64), m0=8, contrasts=(10.0, 100.0), count=4096,
                        tol=1e-10),
    "adjoint_L64": dict(L=64, m0=16, contrast=100.0, count=64, tol=1e-13),
    "large_L256": dict(L=256, m0=8, contrast=100.0, count=256, tol=1e-10),
}


def config_batch(name: str, seed: int = 0, count: int | None = None, start: int = 0) -> list:
    """Descriptors of configuration `name` (optionally only `count` of them)."""
    c = CONFIGS[name]
    cnt = c["count"] if count is None else int(count)
    if name == "uneven_4096":
        g = np.random.default_rng(seed)
        Ls = g.choice(np.asarray(c["Ls"]), size=c["count"])
        lam = g.choice(np.asarray(c["contrasts"]), size=c["count"])
        return [realization(int(Ls[k]), c["m0"], float(lam[k]), seed, k)
                for k in range(start, start + cnt)]
    return batch(c["L"], c["m0"], c["contrast"], seed, cnt, start=start)


def fd_cells(n: int, count: int, seed: int, index: int) -> np.ndarray:
    """`count` distinct random cells (c1, c2) of an n x n grid for finite-difference checks."""
    g = np.random.default_rng([seed, index, 7])
    flat = g.choice(n * n, size=count, replace=False)
    return np.stack([flat // n, flat % n], axis=1)
