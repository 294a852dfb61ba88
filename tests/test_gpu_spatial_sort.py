"""Spatial sort (options.spatial_sort): the context stores atoms in cell order, while every
input and output stays in the caller's order. On a shuffled input the sorted context gives
the oracle's lists bit-exactly and its charges, forces and energies within the parity
tolerances, and the unsorted context's molecules, trajectory and (after resort) state."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rx():
    from paper_1706_07772_gb300 import build as B
    B.build()
    import paper_1706_07772_gb300.reaxff as m
    m.load()
    return m


def shuffled(name, seed=5):
    w = synth.workload(name)
    p = np.random.default_rng(seed).permutation(len(w["x"]))
    return dict(w, types=w["types"][p], x=w["x"][p], v=w["v"][p])


def keyset(i, j, s, n):
    return np.sort(oracle.sort_key(np.asarray(i, np.int64), np.asarray(j, np.int64), np.asarray(s, np.int64), n))


@pytest.mark.parametrize("name", ["petn464", "cluster300"])
def test_sorted_context_matches_oracle_in_callers_order(rx, params, name):
    w = shuffled(name)
    n = len(w["x"])
    o = dict(w["options"], qeq_tol=1e-10)
    m = oracle.Model(params, w["types"], w["box"], o)
    ref = m.forces(w["x"], tol=1e-10)
    c = rx.ReaxFF(params, w["types"], w["box"], o, precision=0, spatial_sort=1)   # QEq to 1e-10 as well
    c.set_state(w["x"], w["v"])
    c.build_lists()
    L = ref["lists"]
    B = L["bond"]
    want = {rx.LIST_FAR: keyset(L["far"]["i"], L["far"]["j"], L["far"]["s"], n),
            rx.LIST_BOND: keyset(np.concatenate([B["i"], B["j"]]), np.concatenate([B["j"], B["i"]]),
                                 np.concatenate([B["s"], -B["s"]]), n),
            rx.LIST_HBOND: keyset(L["hbond"]["i"], L["hbond"]["j"], L["hbond"]["s"], n)}
    for which, k in want.items():
        assert np.array_equal(keyset(*c.get_lists(which), n), k), which
    q, _, _, conv = c.qeq()
    assert conv and np.abs(q - ref["qeq"]["q"]).max() < 1e-8
    F, E, W = c.forces(q=ref["qeq"]["q"])
    rms = np.sqrt((ref["F"] ** 2).mean())
    assert np.abs(F - ref["F"]).max() / rms < 1e-9
    assert abs(E[0].sum() - ref["E_total"]) < 1e-10 * abs(ref["E_total"])
    # bond orders come in the entry order of the bond list
    i, j, s = c.get_lists(rx.LIST_BOND)
    bo = c.get_bond_orders()["bo"]
    okey = oracle.sort_key(B["i"], B["j"], B["s"], n)
    pos = {k: t for t, k in enumerate(okey)}
    canon = oracle.half_mask(i, j, s)
    gkey = oracle.sort_key(i[canon].astype(np.int64), j[canon].astype(np.int64), s[canon].astype(np.int64), n)
    assert np.allclose(bo[canon], ref["parts"]["bo"][np.array([pos[k] for k in gkey])], rtol=1e-12, atol=1e-15)
    c.close()


def test_sorted_and_unsorted_contexts_agree(rx, params):
    """Same shuffled input, FP64: molecules identical (numbered by smallest caller index),
    MD trajectories equal to rounding, and resort keeps the state bit for bit."""
    w = shuffled("petn464", seed=9)
    ctx = {}
    for srt in (0, 1):
        c = rx.ReaxFF(params, w["types"], w["box"], w["options"], precision=0, spatial_sort=srt)
        c.set_state(w["x"], w["v"])
        ctx[srt] = c
    mol0, sp0 = ctx[0].species()
    mol1, sp1 = ctx[1].species()
    assert np.array_equal(mol0, mol1) and sp0 == sp1
    e0 = ctx[0].step(10, 0.1)
    e1 = ctx[1].step(10, 0.1)
    x0, v0, q0 = ctx[0].get_state()
    x1, v1, q1 = ctx[1].get_state()
    assert np.abs(x1 - x0).max() < 1e-9 and np.abs(v1 - v0).max() < 1e-9
    assert np.abs(q1 - q0).max() < 1e-7
    assert np.abs(e1 - e0).max() < 1e-9 * np.abs(e0).max()
    ctx[1].resort()
    x2, v2, _ = ctx[1].get_state()
    assert np.array_equal(x2, x1) and np.array_equal(v2, v1)
    e0b = ctx[0].step(5, 0.1)
    e1b = ctx[1].step(5, 0.1)
    x0, _, _ = ctx[0].get_state()
    x1, _, _ = ctx[1].get_state()
    assert np.abs(x1 - x0).max() < 1e-9
    assert np.abs(e1b - e0b).max() < 1e-9 * np.abs(e0b).max()
    for c in ctx.values():
        c.close()
