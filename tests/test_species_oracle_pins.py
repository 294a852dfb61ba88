"""Pins of the species-analysis oracle: hand-built bond graphs, an independent BFS,
permutation invariance -- no GPU."""
import numpy as np

from oracle import species_oracle as so


def test_hand_built_graph():
    # 0-1-2 (C, O, O) connected; 3-4 (H, H) with a bond exactly at the threshold (not
    # bonded: strict >); 5 alone (N); 6-7 via a periodic image entry counted once each way
    types = np.array([0, 3, 3, 1, 1, 2, 0, 0])
    bi = np.array([0, 1, 3, 6, 7])
    bj = np.array([1, 2, 4, 7, 6])
    bo = np.array([0.9, 1.2, 0.3, 0.5, 0.5])
    mol, m = so.molecules(8, bi, bj, bo, types)
    assert m == 5
    assert list(mol) == [0, 0, 0, 1, 2, 3, 4, 4]
    sp = so.species(types, mol, m)
    assert sp == {(0, 1, 0, 0, 2): 1, (0, 0, 1, 0, 0): 2, (0, 0, 0, 1, 0): 1, (0, 2, 0, 0, 0): 1}


def test_union_find_equals_bfs_and_is_permutation_invariant():
    rng = np.random.default_rng(4)
    n = 300
    types = rng.integers(0, 4, n)
    bi = rng.integers(0, n, 700)
    bj = rng.integers(0, n, 700)
    bo = rng.uniform(0, 0.9, 700)
    thr = rng.uniform(0.2, 0.5, (4, 4))
    m1, k1 = so.molecules(n, bi, bj, bo, types, thr)
    m2, k2 = so.molecules_bfs(n, bi, bj, bo, types, thr)
    assert k1 == k2 and np.array_equal(m1, m2)
    # relabel the atoms: the species histogram does not change
    p = rng.permutation(n)
    inv = np.empty(n, int)
    inv[p] = np.arange(n)
    m3, k3 = so.molecules(n, inv[bi], inv[bj], bo, types[p], thr)
    assert k3 == k1
    assert so.species(types[p], m3, k3) == so.species(types, m1, k1)


def test_counts_sum_to_atoms():
    rng = np.random.default_rng(1)
    n = 50
    types = rng.integers(0, 4, n)
    bi, bj = rng.integers(0, n, 60), rng.integers(0, n, 60)
    mol, m = so.molecules(n, bi, bj, np.ones(60), types)
    sp = so.species(types, mol, m)
    assert sum(sum(k[1:]) * v for k, v in sp.items()) == n
    assert sum(sp.values()) == m
