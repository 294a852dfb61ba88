"""Seeded synthetic CHNO molecular crystal (input generator only).

The paper benchmarks on a PETN crystal (Sec. 4, PETN crystal benchmark) whose deck is
not available. This module builds a stand-in with the same composition and density:
a tetragonal cell a = b = 9.38 A, c = 6.71 A holding two C5H8N4O12 molecules (58
atoms), each made from generic bond geometry (a central C with four CH2-O-NO2 arms)
and placed at fractional (0,0,0) and (1/2,1/2,1/2) with seeded orientations.
No published crystal coordinates are used.

This module holds none of the ReaxFF arithmetic: it only produces types, positions,
velocities and boxes, and is shared by the oracle and the CUDA path as input.
"""
from __future__ import annotations

import numpy as np

C, H, N, O = 0, 1, 2, 3
TYPE_NAMES = ("C", "H", "N", "O")
MASS = np.array([12.011, 1.008, 14.007, 15.999])
CELL = np.array([9.38, 9.38, 6.71])
KB = 0.0019872041           # kcal/(mol K)
ACC_CONV = 4.184e-4          # (kcal/mol/A)/amu -> A/fs^2

# generic bond lengths (A)
_CC, _CH, _CO, _ON, _NO = 1.54, 1.09, 1.44, 1.40, 1.21


def _place(a, b, c, bond, angle, dihedral):
    """Position d with |cd| = bond, angle(b,c,d) = angle, dihedral(a,b,c,d) = dihedral (rad)."""
    bc = c - b
    bc /= np.linalg.norm(bc)
    n = np.cross(b - a, bc)
    n /= np.linalg.norm(n)
    m = np.cross(n, bc)
    d2 = np.array([-bond * np.cos(angle),
                   bond * np.sin(angle) * np.cos(dihedral),
                   bond * np.sin(angle) * np.sin(dihedral)])
    return c + d2[0] * bc + d2[1] * m + d2[2] * n


def _perp_frame(d):
    t = np.array([1.0, 0.0, 0.0]) if abs(d[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    u = np.cross(d, t)
    u /= np.linalg.norm(u)
    w = np.cross(d, u)
    return u, w


def molecule(phis, psis):
    """One C(CH2-O-NO2)4 molecule: 29 atoms. phis/psis: arm twist angles (rad)."""
    tet = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float) / np.sqrt(3.0)
    types = [C]
    xyz = [np.zeros(3)]
    for k, d in enumerate(tet):
        c1 = _CC * d
        u, w = _perp_frame(d)

        def tdir(phi):
            return d / 3.0 + (2.0 * np.sqrt(2.0) / 3.0) * (np.cos(phi) * u + np.sin(phi) * w)

        o1 = c1 + _CO * tdir(phis[k])
        h1 = c1 + _CH * tdir(phis[k] + 2.0 * np.pi / 3.0)
        h2 = c1 + _CH * tdir(phis[k] + 4.0 * np.pi / 3.0)
        n1 = _place(np.zeros(3), c1, o1, _ON, np.deg2rad(112.0), psis[k])
        o2 = _place(c1, o1, n1, _NO, np.deg2rad(118.0), 0.0)
        o3 = _place(c1, o1, n1, _NO, np.deg2rad(118.0), np.pi)
        types += [C, H, H, O, N, O, O]
        xyz += [c1, h1, h2, o1, n1, o2, o3]
    return np.array(types, np.int32), np.array(xyz)


def _rand_rot(rng, scale=None):
    """Uniform random rotation (or a small one of angle ~scale rad)."""
    if scale is None:
        q = rng.normal(size=4)
    else:
        q = np.concatenate([[1.0], rng.normal(scale=0.5 * scale, size=3)])
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a*a+b*b-c*c-d*d, 2*(b*c-a*d), 2*(b*d+a*c)],
                     [2*(b*c+a*d), a*a-b*b+c*c-d*d, 2*(c*d-a*b)],
                     [2*(b*d-a*c), 2*(c*d+a*b), a*a-b*b-c*c+d*d]])


_SHIFTS = np.array([[sx, sy, sz] for sx in (-1, 0, 1) for sy in (-1, 0, 1) for sz in (-1, 0, 1)], float)


def _bond_hops(nat=29):
    """Topological distance (bond hops) inside one molecule, from the build order."""
    g = np.full((nat, nat), 99, int)
    np.fill_diagonal(g, 0)
    edges = []
    for k in range(4):
        b = 1 + 7 * k            # c1, h1, h2, o1, n1, o2, o3
        edges += [(0, b), (b, b + 1), (b, b + 2), (b, b + 3), (b + 3, b + 4), (b + 4, b + 5), (b + 4, b + 6)]
    for i, j in edges:
        g[i, j] = g[j, i] = 1
    for k in range(nat):
        g = np.minimum(g, g[:, k:k + 1] + g[k:k + 1, :])
    return g


_HOPS = _bond_hops()


def _contact(mols):
    """Smallest distance between atoms that are not within 2 bonds of each other."""
    xs = np.concatenate([x for _, x in mols])
    nm = len(mols)
    nat = mols[0][1].shape[0]
    d = xs[None, :, None, :] - xs[:, None, None, :] + _SHIFTS[None, None, :, :] * CELL
    r = np.sqrt((d * d).sum(-1))                      # (n, n, 27)
    same = np.zeros((nm * nat, nm * nat), bool)
    for m in range(nm):
        same[m * nat:(m + 1) * nat, m * nat:(m + 1) * nat] = _HOPS <= 2
    r[:, :, 13] = np.where(same, np.inf, r[:, :, 13])
    idx = np.arange(nm * nat)
    r[idx, idx, :] = np.where(np.arange(27)[None, :] == 13, np.inf, r[idx, idx, :])
    return float(r.min())


def _build(params):
    mols = []
    for centre, (rot, phis, psis) in zip((np.zeros(3), 0.5 * CELL), params):
        t, x = molecule(phis, psis)
        mols.append((t, x @ rot.T + centre))
    return mols


def search_unit_cell(seed: int = 1706, trials: int = 400, refine: int = 3000, accept: float = 2.2):
    """Seeded search for a 58-atom cell; returns (types, xyz, min_contact).

    Orientations and arm twists are drawn at random, the best draw is refined by a
    seeded hill climb on the smallest non-bonded contact (intra- and intermolecular,
    periodic), stopping once the contact reaches `accept` A.
    """
    rng = np.random.default_rng(seed)
    best, best_p = -1.0, None
    for _ in range(trials):
        p = [(_rand_rot(rng), rng.uniform(0, 2 * np.pi, 4), rng.uniform(0, 2 * np.pi, 4)) for _ in range(2)]
        c = _contact(_build(p))
        if c > best:
            best, best_p = c, p
    step = 0.3
    for it in range(refine):
        if best >= accept + 0.05:
            break
        p = [(_rand_rot(rng, step) @ rot, phis + rng.normal(scale=step, size=4), psis + rng.normal(scale=step, size=4))
             for rot, phis, psis in best_p]
        c = _contact(_build(p))
        if c > best:
            best, best_p = c, p
        if it % 500 == 499:
            step *= 0.7
    mols = _build(best_p)
    types = np.concatenate([t for t, _ in mols])
    xyz = np.concatenate([x for _, x in mols])
    return types, xyz, best


_CELL_FILE = __import__("os").path.join(__import__("os").path.dirname(__file__), "cell58.txt")


def unit_cell():
    """The 58-atom cell written by `python -m synth.make_cell` (seeded search above)."""
    rows = np.loadtxt(_CELL_FILE, comments="#")
    return rows[:, 0].astype(np.int32), rows[:, 1:4].copy()


def crystal(ncell, seed: int = 0, jitter: float = 0.05):
    """Replicate the cell ncell = (nx, ny, nz) times; seeded Gaussian jitter (A).

    Returns (types int32[n], x float64[n,3] wrapped into [0, L), box float64[3]).
    Atoms are ordered cell by cell (x fastest), which keeps them spatially local.
    """
    t0, x0 = unit_cell()
    nx, ny, nz = ncell
    box = CELL * np.array([nx, ny, nz], float)
    shifts = np.array([[ix, iy, iz] for iz in range(nz) for iy in range(ny) for ix in range(nx)], float) * CELL
    x = (shifts[:, None, :] + x0[None, :, :]).reshape(-1, 3)
    types = np.tile(t0, len(shifts)).astype(np.int32)
    rng = np.random.default_rng(seed)
    x = x + rng.normal(scale=jitter, size=x.shape)
    x = np.mod(x, box)
    x[x >= box] -= box[np.nonzero(x >= box)[1]]
    return types, x, box


def velocities(types, temperature: float, seed: int = 0):
    """Maxwell-Boltzmann velocities (A/fs) at exactly `temperature` K over 3n-3 DoF.

    Gaussian N(0, kT/m) per component, centre-of-mass momentum removed, then rescaled.
    """
    n = len(types)
    m = MASS[types]
    rng = np.random.default_rng(seed)
    sig = np.sqrt(KB * temperature * ACC_CONV / m)
    v = rng.normal(size=(n, 3)) * sig[:, None]
    v -= (m[:, None] * v).sum(0) / m.sum()
    ke = 0.5 * (m[:, None] * v * v).sum() / ACC_CONV
    t_now = 2.0 * ke / ((3 * n - 3) * KB)
    return v * np.sqrt(temperature / t_now)


def random_cluster(n: int, box, seed: int = 0, dmin: float = 0.95, fractions=(0.3, 0.3, 0.15, 0.25)):
    """Random dense CHNO configuration (test input rich in every interaction kind).

    Atoms are placed uniformly with rejection below `dmin` A (periodic), types drawn
    with the given C/H/N/O fractions.
    """
    rng = np.random.default_rng(seed)
    box = np.asarray(box, float)
    x = np.zeros((0, 3))
    while len(x) < n:
        p = rng.uniform(0, 1, 3) * box
        if len(x):
            d = x - p
            d -= box * np.round(d / box)
            if (d * d).sum(1).min() < dmin * dmin:
                continue
        x = np.vstack([x, p])
    types = rng.choice(4, size=n, p=np.asarray(fractions) / np.sum(fractions)).astype(np.int32)
    return types, x, box
