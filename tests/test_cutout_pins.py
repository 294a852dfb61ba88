"""Pins of the cut-out evaluation of the oracle (oracle/cutout.py), used by the full-size GPU
parity tests, against the whole periodic oracle on a crystal small enough to evaluate in full
(4x4x6 cells, 5,568 atoms, fixed seeded charges)."""
import numpy as np
import pytest

import oracle
import synth
from oracle import cutout
from synth.crystal import crystal
from synth.workloads import OPTIONS_DEFAULT


@pytest.fixture(scope="module")
def system():
    P = synth.make_params()
    types, x, box = crystal((4, 4, 6), seed=3)
    box = np.asarray(box, float)
    opts = dict(OPTIONS_DEFAULT)
    rng = np.random.default_rng(5)
    q = rng.normal(0.0, 0.3, len(x))
    q -= q.mean()
    m = oracle.Model(P, types, box, opts)
    full = m.forces(x, q=q)
    return dict(P=P, types=types, x=x, box=box, opts=opts, q=q, m=m, full=full, rng=rng)


def _key(i, j, s, n):
    return np.sort(oracle.sort_key(np.asarray(i, np.int64), np.asarray(j, np.int64), np.asarray(s, np.int64), n))


def test_bond_reach_bounds_every_bond(system):
    """The reach is where BO' falls below bo_cut for every pair (and not 50 um earlier for
    some pair), and no bond of the crystal is longer."""
    P, o = system["P"], system["opts"]
    b = cutout.bond_reach(P, o)
    assert 0.0 < b < o["r_bond"]
    nt = np.asarray(P["r0s"]).shape[0]
    tot = lambda r: max(sum(oracle.reaxff_oracle.bo_prime_np(np.array([r]), np.array([a]), np.array([c]), P, o["bo_cut"]))[0]
                        for a in range(nt) for c in range(nt))
    assert tot(b) < o["bo_cut"] <= tot(b - 5e-5)
    B = system["full"]["lists"]["bond"]
    d = (system["x"][B["j"]] - system["x"][B["i"]]) + B["s"] * system["box"]
    assert np.sqrt((d * d).sum(1)).max() < b
    assert cutout.dependency_radius(P, o) == max(6 * b, o["r_hb"] + 2 * b, o["r_nb"])


def test_cutout_forces_equal_whole_system(system):
    """Forces on sampled atoms from the cut-out equal the whole periodic system's; a cut-out
    6 A deep (well below the dependency radius) does not, so the comparison has teeth."""
    s = system
    F = s["full"]["F"]
    rms = np.sqrt((F ** 2).mean())
    D = cutout.dependency_radius(s["P"], s["opts"])
    for a in s["rng"].choice(len(s["x"]), 3, replace=False):
        c = s["x"][a]
        ids, rr = cutout.region(s["x"], s["box"], c, 4)
        cu = cutout.Cutout(s["P"], s["types"], s["x"], s["box"], s["opts"], c, rr + D)
        assert np.abs(cu.forces(s["q"], ids) - F[ids]).max() < 1e-11 * rms
    c = s["x"][0]
    ids, rr = cutout.region(s["x"], s["box"], c, 4)
    thin = cutout.Cutout(s["P"], s["types"], s["x"], s["box"], s["opts"], c, rr + 6.0)
    assert np.abs(thin.forces(s["q"], ids) - F[ids]).max() > 1e-4 * rms


def test_list_rows_equal_whole_system_lists(system):
    """Far, bond (both directions) and H-bond rows of sampled atoms, decided on the global
    coordinates, equal the rows of the whole system's lists as sets."""
    s = system
    n = len(s["x"])
    L = s["full"]["lists"]
    B = L["bond"]
    full = dict(far=(L["far"]["i"], L["far"]["j"], L["far"]["s"]),
                bond=(np.concatenate([B["i"], B["j"]]), np.concatenate([B["j"], B["i"]]),
                      np.concatenate([B["s"], -B["s"]])),
                hbond=(L["hbond"]["i"], L["hbond"]["j"], L["hbond"]["s"]))
    hflag = np.asarray(s["P"]["hb"])[s["types"]] == 1
    # rows around an H atom so that H-bond rows are present
    seen = dict(far=0, bond=0, hbond=0)
    for c in (s["x"][np.nonzero(hflag)[0][7]], s["x"][11]):
        ids, rr = cutout.region(s["x"], s["box"], c, 6)
        cu = cutout.Cutout(s["P"], s["types"], s["x"], s["box"], s["opts"], c, rr + s["opts"]["r_nb"] + 1.0)
        R = cutout.list_rows(s["x"], s["types"], s["box"], s["P"], s["opts"], ids, cu.ids)
        for k, (i, j, sh) in full.items():
            sel = np.isin(i, ids)
            assert np.array_equal(_key(i[sel], j[sel], sh[sel], n), _key(R[k]["i"], R[k]["j"], R[k]["s"], n)), k
            seen[k] += len(R[k]["i"])
    assert min(seen.values()) > 0, seen


def test_qeq_rows_give_the_chemical_potential(system):
    """At the converged QEq charges of the whole system, chi_i + (H q)_i from the cut-out
    equals the common mu (optimality of the constrained minimum) and the whole system's
    own row products."""
    s = system
    L = s["full"]["lists"]
    qq = s["m"].qeq(s["x"], L, tol=1e-13, max_iter=2000)
    Hm = s["m"].qeq_matrix(s["x"], L)
    chi = np.asarray(s["P"]["chi"])[s["types"]]
    c = s["x"][100]
    ids, rr = cutout.region(s["x"], s["box"], c, 16)
    cu = cutout.Cutout(s["P"], s["types"], s["x"], s["box"], s["opts"], c, rr + s["opts"]["r_nb"] + 1.0)
    rho, mag = cu.qeq_rows(qq["q"], ids)
    whole = chi[ids] + Hm[ids] @ qq["q"]
    assert np.abs(rho - whole).max() < 1e-12 * mag.max()
    assert np.abs(rho - qq["mu"]).max() < 1e-9 * (abs(qq["mu"]) + np.abs(chi).max())
    assert np.all(mag >= np.abs(rho - chi[ids]))
