"""In-situ species analysis (Sec. 3.4) on the GPU against the oracle
(oracle/species_oracle.py) on the oracle's own bond orders."""
import numpy as np
import pytest

import oracle
import synth
from oracle import species_oracle as so

pytestmark = pytest.mark.gpu

_REF = {}


def _ref(params, name):
    if name not in _REF:
        w = synth.workload(name)
        o = dict(w["options"], qeq_tol=1e-10)
        m = oracle.Model(params, w["types"], w["box"], o)
        r = m.forces(w["x"], tol=1e-10)
        _REF[name] = (w, o, r["lists"]["bond"], r["parts"]["bo"])
    return _REF[name]


@pytest.fixture(scope="module")
def rx():
    import paper_1706_07772_gb300.reaxff as rx
    rx.load()
    return rx


def _thr_table(rng=None):
    if rng is None:
        return None
    t = np.full((8, 8), 0.3)
    t[:4, :4] = rng.uniform(0.15, 0.6, (4, 4))
    return (t + t.T) / 2.0


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", ["petn464", "cluster300"])
@pytest.mark.parametrize("custom", [False, True])
def test_species_match_oracle(rx, params, name, prec, custom):
    w, o, B, bo = _ref(params, name)
    types = np.asarray(w["types"])
    thr = _thr_table(np.random.default_rng(3)) if custom else None
    t4 = np.full((4, 4), 0.3) if thr is None else thr[:4, :4]
    # no bond order within the GPU path's error of a threshold (else the sets may differ)
    margin = 1e-9 if prec == 0 else 1e-4
    assert np.all(np.abs(bo - t4[types[B["i"]], types[B["j"]]]) > margin)
    mol_ref, m_ref = so.molecules(len(types), B["i"], B["j"], bo, types, t4)
    sp_ref = so.species(types, mol_ref, m_ref)
    c = rx.ReaxFF(params, w["types"], w["box"], o, precision=prec)
    c.set_state(w["x"], w["v"])
    c.forces()
    mol, sp = c.species(thr)
    assert np.array_equal(mol, mol_ref)
    got = {(k[0],) + k[1:5]: v for k, v in sp.items()}
    assert all(sum(k[5:]) == 0 for k in sp)                   # types 4..7 absent
    assert got == dict(sp_ref)
    c.close()


def test_species_per_replica(rx, params):
    specs = [("petn464", 0), ("cluster300", 1), ("petn464", 2)]
    ws = [synth.workload(nm, seed=sd) for nm, sd in specs]
    types = np.concatenate([w["types"] for w in ws])
    x = np.concatenate([w["x"] for w in ws])
    off = np.cumsum([0] + [len(w["x"]) for w in ws])
    boxes = np.stack([w["box"] for w in ws])
    o = dict(ws[0]["options"], qeq_tol=1e-10)
    cb = rx.ReaxFF(params, types, boxes, o, precision=0, rep_offsets=off)
    cb.set_state(x)
    cb.forces()
    mol_b, sp_b = cb.species()
    for r, w in enumerate(ws):
        c = rx.ReaxFF(params, w["types"], w["box"], o, precision=0)
        c.set_state(w["x"])
        c.forces()
        mol, sp = c.species()
        mine = {k[1:]: v for k, v in sp_b.items() if k[0] == r}
        assert mine == {k[1:]: v for k, v in sp.items()}
        # molecules never cross replicas; numbering follows the smallest atom index
        mb = mol_b[off[r]:off[r + 1]]
        assert np.array_equal(mb - mb.min(), mol - mol.min())
        c.close()
    cb.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_time_averaged_bond_orders_and_species(rx, params, prec):
    """Four samples at host-made positions (the crystal with seeded 0.03 A displacements):
    the averaged bond order of every directed pair seen equals the oracle's average of its
    own bond orders, and the species analysis on the averages matches the oracle's."""
    w = synth.workload("petn464")
    types = np.asarray(w["types"])
    box = np.asarray(w["box"], float)
    o = dict(w["options"], qeq_tol=1e-10)
    rng = np.random.default_rng(5)
    xs = [np.mod(w["x"] + rng.normal(scale=0.03, size=w["x"].shape), box) for _ in range(4)]
    m = oracle.Model(params, types, box, o)
    samples = []
    for x in xs:
        r = m.forces(x, tol=1e-10)
        B, bo = r["lists"]["bond"], r["parts"]["bo"]
        samples.append((np.concatenate([B["i"], B["j"]]), np.concatenate([B["j"], B["i"]]),
                        np.concatenate([B["s"], -B["s"]]), np.concatenate([bo, bo])))
    ref = so.average_bond_orders(samples)
    c = rx.ReaxFF(params, w["types"], w["box"], o, precision=prec)
    c.bo_average_reset()
    for x in xs:
        c.set_state(x, w["v"])
        c.bo_average_sample()
    assert c.bo_average_samples() == 4
    i, j, s, a = c.get_bo_average()
    got = {(int(p), int(q), int(t[0]), int(t[1]), int(t[2])): float(v) for p, q, t, v in zip(i, j, s, a)}
    assert set(got) == set(ref)
    tol = 1e-9 if prec == 0 else 2e-6
    assert max(abs(got[k] - ref[k]) for k in ref) < tol
    keys = sorted(ref)
    avg = np.array([ref[k] for k in keys])
    ki = np.array([k[0] for k in keys])
    kj = np.array([k[1] for k in keys])
    margin = 1e-9 if prec == 0 else 1e-4
    assert np.all(np.abs(avg - 0.3) > margin)
    mol_ref, m_ref = so.molecules(len(types), ki, kj, avg, types)
    mol, sp = c.species_average()
    assert np.array_equal(mol, mol_ref)
    got_sp = {(k[0],) + k[1:5]: v for k, v in sp.items()}
    assert got_sp == dict(so.species(types, mol_ref, m_ref))
    c.bo_average_reset()
    assert c.bo_average_samples() == 0
    with pytest.raises(rx.ReaxFFError):
        c.species_average()
    c.close()
