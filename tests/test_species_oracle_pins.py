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


def test_time_average_hand_built():
    """Averages by hand: a persistent pair (0.2, 0.4, 0.6 -> 0.4), a transient one seen in
    one of three samples (0.9 -> 0.3), image shifts kept apart; one sample is itself."""
    z = np.zeros((1, 3), int)
    e = np.array([[1, 0, 0]])
    samples = [
        (np.array([0, 2]), np.array([1, 3]), np.array([[0, 0, 0], [0, 0, 0]]), np.array([0.2, 0.9])),
        (np.array([0]), np.array([1]), z, np.array([0.4])),
        (np.array([0, 0]), np.array([1, 1]), np.concatenate([z, e]), np.array([0.6, 0.75])),
    ]
    avg = so.average_bond_orders(samples)
    assert set(avg) == {(0, 1, 0, 0, 0), (2, 3, 0, 0, 0), (0, 1, 1, 0, 0)}
    assert abs(avg[(0, 1, 0, 0, 0)] - 0.4) < 1e-15
    assert abs(avg[(2, 3, 0, 0, 0)] - 0.3) < 1e-15
    assert abs(avg[(0, 1, 1, 0, 0)] - 0.25) < 1e-15
    one = so.average_bond_orders(samples[:1])
    assert one == {(0, 1, 0, 0, 0): 0.2, (2, 3, 0, 0, 0): 0.9}


def test_transient_encounter_is_not_a_bond_after_averaging():
    """An encounter at BO 0.9 in one of four samples averages to 0.225 < 0.3: the two atoms
    stay separate molecules, while a bond at 0.35 in every sample joins its atoms."""
    types = np.array([0, 1, 0, 1])
    samples = []
    for k in range(4):
        bi, bj, bo = [0, 1], [1, 0], [0.35, 0.35]
        if k == 2:
            bi, bj, bo = bi + [2, 3], bj + [3, 2], bo + [0.9, 0.9]
        samples.append((np.array(bi), np.array(bj), np.zeros((len(bi), 3), int), np.array(bo)))
    avg = so.average_bond_orders(samples)
    keys = sorted(avg)
    mol, m = so.molecules(4, [k[0] for k in keys], [k[1] for k in keys], [avg[k] for k in keys], types)
    assert m == 3 and list(mol) == [0, 0, 1, 2]
    inst, mi = so.molecules(4, samples[2][0], samples[2][1], samples[2][3], types)
    assert mi == 2 and list(inst) == [0, 0, 1, 1]          # the instant alone joins 2 and 3
