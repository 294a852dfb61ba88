"""Named synthetic workloads (sizes of the paper's PETN benchmark stand-in).

  petn464      2x2x2 cells,   464 atoms, box 18.76 x 18.76 x 13.42 A, QEq tol 1e-8
  petn32k      10x8x7 cells,  32,480 atoms, box 93.80 x 75.04 x 46.97 A, QEq tol 1e-6
  petn1m       32x28x20 cells, 1,039,360 atoms, box 300.16 x 262.64 x 134.20 A, tol 1e-6
  batch64      64 replicas, 2x2x2 ... 8x4x4 cells (seeded shapes), 250-350 K
  cluster<n>   random dense CHNO configuration (tests only)
"""
from __future__ import annotations

import numpy as np

from synth.crystal import crystal, random_cluster, velocities

OPTIONS_DEFAULT = dict(r_nb=10.0, r_bond=5.0, r_hb=7.5, bo_cut=1e-3, thb_cut=1e-3,
                       thb_cutsq=1e-5, hb_bo_min=0.01, qeq_tol=1e-6, qeq_max_iter=200)

_CELLS = {"petn464": (2, 2, 2), "petn32k": (10, 8, 7), "petn1m": (32, 28, 20)}


def workload(name: str, seed: int = 0, temperature: float = 300.0):
    """Return dict(types, x, v, box, options) for a named single-system workload."""
    opts = dict(OPTIONS_DEFAULT)
    if name in _CELLS:
        types, x, box = crystal(_CELLS[name], seed=seed)
        if name == "petn464":
            opts["qeq_tol"] = 1e-8
    elif name.startswith("cluster"):
        n = int(name[len("cluster"):])
        side = (n / 0.075) ** (1.0 / 3.0)
        types, x, box = random_cluster(n, (side, side, side), seed=seed)
    else:
        raise ValueError(name)
    v = velocities(types, temperature, seed=seed + 1)
    return dict(types=types, x=x, v=v, box=np.asarray(box, float), options=opts)


def fixed_charges(n: int, seed: int = 0, scale: float = 0.3):
    """Seeded neutral charges (e) for evaluating forces at fixed charges: normal with standard
    deviation `scale`, shifted to zero sum."""
    q = np.random.default_rng(seed).normal(0.0, scale, n)
    return q - q.mean()


def batch_shapes(nrep: int = 64, seed: int = 0):
    """Seeded uneven replica shapes from 2x2x2 to 8x4x4 cells and temperatures 250-350 K."""
    rng = np.random.default_rng(seed)
    shapes = [(2, 2, 2), (8, 4, 4)]
    while len(shapes) < nrep:
        shapes.append((int(rng.integers(2, 9)), int(rng.integers(2, 5)), int(rng.integers(2, 5))))
    temps = rng.uniform(250.0, 350.0, nrep)
    return shapes, temps
