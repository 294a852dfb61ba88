"""FP64 CPU oracle of the in-situ molecular species analysis -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU legs may import this module. It
shares no code with the CUDA path.

Sec. 3.4: two atoms are bonded when the bond order between them exceeds a threshold for
their pair of elements (default 0.3); the molecule ID of an atom is the smallest atom ID
of its connected component in that bond graph; molecule IDs are renumbered 0..M-1 in the
order of those smallest IDs; a species is the vector of atom counts per element of a
molecule (isomers are not distinguished); the summary is the count of molecules of each
species (per replica of a batch). The bond orders may be time averages over samples
(average_bond_orders), so that transient encounters do not count as bonds.
"""
from __future__ import annotations

from collections import Counter

import numpy as np

NT = 4


def molecules(n, bi, bj, bo, types, thr=None):
    """Molecule index (0..M-1, ordered by the smallest atom of each molecule) of every atom,
    by union-find over the bonds with bo > thr[type_i, type_j]."""
    thr = np.full((NT, NT), 0.3) if thr is None else np.asarray(thr, float)
    parent = list(range(n))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for i, j, b in zip(np.asarray(bi), np.asarray(bj), np.asarray(bo)):
        if b > thr[types[i], types[j]]:
            ra, rb = find(int(i)), find(int(j))
            if ra != rb:
                parent[max(ra, rb)] = min(ra, rb)
    root = np.array([find(a) for a in range(n)])
    roots = np.unique(root)                    # sorted: smallest member order
    return np.searchsorted(roots, root), len(roots)


def molecules_bfs(n, bi, bj, bo, types, thr=None):
    """The same by breadth-first search from each unvisited atom in index order (an
    independent restatement of the definition, used to pin molecules())."""
    thr = np.full((NT, NT), 0.3) if thr is None else np.asarray(thr, float)
    adj = [[] for _ in range(n)]
    for i, j, b in zip(np.asarray(bi), np.asarray(bj), np.asarray(bo)):
        if b > thr[types[i], types[j]]:
            adj[int(i)].append(int(j))
            adj[int(j)].append(int(i))
    mol = np.full(n, -1)
    m = 0
    for s in range(n):
        if mol[s] >= 0:
            continue
        mol[s] = m
        todo = [s]
        while todo:
            a = todo.pop()
            for b in adj[a]:
                if mol[b] < 0:
                    mol[b] = m
                    todo.append(b)
        m += 1
    return mol, m


def average_bond_orders(samples):
    """Time-averaged bond orders (Sec. 3.4: bonds judged on bond orders averaged over
    samples). samples: one (i, j, shift (m, 3), bo) tuple of directed bond entries per
    sample. Returns {(i, j, sx, sy, sz): (sum of bo over the samples) / (number of
    samples)} over every pair seen; a pair missing from a sample contributes 0."""
    acc = {}
    for i, j, sh, bo in samples:
        for a, b, s3, v in zip(np.asarray(i), np.asarray(j), np.asarray(sh), np.asarray(bo)):
            key = (int(a), int(b), int(s3[0]), int(s3[1]), int(s3[2]))
            acc[key] = acc.get(key, 0.0) + float(v)
    return {k: v / len(samples) for k, v in acc.items()}


def species(types, mol, m, rep=None):
    """Counter {(replica, nC, nH, nN, nO): molecules}."""
    types = np.asarray(types)
    rep = np.zeros(len(types), int) if rep is None else np.asarray(rep)
    cnt = np.zeros((m, NT), int)
    np.add.at(cnt, (mol, types), 1)
    mrep = np.zeros(m, int)
    mrep[mol] = rep
    return Counter((int(mrep[k]),) + tuple(int(c) for c in cnt[k]) for k in range(m))
