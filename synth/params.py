"""Seeded synthetic 4-element (C, H, N, O) ReaxFF-form parameter set (input generator).

The paper's force-field file is not available and no published parameter values are
used: every value is drawn from a physical range with a fixed seed. Per-pair, per-triple
and per-torsion tables are filled here (combining rules included), so that the method's
code on either side only reads tables.

Units: energy kcal/mol, length A, charge e, mass amu, angles rad.
Layout (all float64 numpy arrays, types 0=C 1=H 2=N 3=O):
  per type   [nt]        mass val vale valboc valang p_lp2 p_ovun2 p_ovun5 p_val3 p_val5
                         chi eta gamma_t hb (int: 0 none, 1 donor H, 2 acceptor)
  per pair   [nt,nt]     r0s r0p r0pp p_bo1..p_bo6 p_boc3 p_boc4 p_boc5 ovc v13 De_s De_p
                         De_pp p_be1 p_be2 p_ovun1 vdw_D vdw_rv vdw_alpha vdw_gw gamma
  per triple [nt,nt,nt]  (i, centre j, k), symmetric in i<->k: th00 p_val1 p_val2 p_val4
                         p_val7 p_pen1 p_coa1
  per torsion[nt,nt]     (centre bond j-k), symmetric: V1 V2 V3 p_tor1 p_cot1
  per hbond  [nt,nt]     (donor-bonded X, acceptor Z): r0hb p_hb1 p_hb2 p_hb3
  general    scalars     p_boc1 p_boc2 p_lp1 p_ovun3 p_ovun4 p_ovun6 p_ovun7 p_ovun8 p_val6
                         p_val8 p_val9 p_val10 p_pen2 p_pen3 p_pen4 p_coa2 p_coa3 p_coa4
                         p_tor2 p_tor3 p_tor4 p_cot2 p_vdW1 k_e
"""
from __future__ import annotations

import numpy as np

from synth.crystal import MASS

NT = 4
PER_TYPE = ("mass", "val", "vale", "valboc", "valang", "p_lp2", "p_ovun2", "p_ovun5",
            "p_val3", "p_val5", "chi", "eta", "gamma_t", "hb")
PER_PAIR = ("r0s", "r0p", "r0pp", "p_bo1", "p_bo2", "p_bo3", "p_bo4", "p_bo5", "p_bo6",
            "p_boc3", "p_boc4", "p_boc5", "ovc", "v13", "De_s", "De_p", "De_pp", "p_be1",
            "p_be2", "p_ovun1", "vdw_D", "vdw_rv", "vdw_alpha", "vdw_gw", "gamma")
PER_TRIPLE = ("th00", "p_val1", "p_val2", "p_val4", "p_val7", "p_pen1", "p_coa1")
PER_TORSION = ("V1", "V2", "V3", "p_tor1", "p_cot1")
PER_HBOND = ("r0hb", "p_hb1", "p_hb2", "p_hb3")
GENERAL = ("p_boc1", "p_boc2", "p_lp1", "p_ovun3", "p_ovun4", "p_ovun6", "p_ovun7",
           "p_ovun8", "p_val6", "p_val8", "p_val9", "p_val10", "p_pen2", "p_pen3", "p_pen4",
           "p_coa2", "p_coa3", "p_coa4", "p_tor2", "p_tor3", "p_tor4", "p_cot2", "p_vdW1", "k_e")

# generic single-bond lengths used for r0 sigma (A): C H N O
_R0 = np.array([[1.54, 1.09, 1.47, 1.43],
                [1.09, 0.80, 1.01, 0.96],
                [1.47, 1.01, 1.45, 1.40],
                [1.43, 0.96, 1.40, 1.48]])


def _sym(rng, lo, hi, nt=NT):
    a = rng.uniform(lo, hi, (nt, nt))
    return np.triu(a) + np.triu(a, 1).T


def make_params(seed: int = 20170623) -> dict:
    """Draw the seeded parameter set (a dict of numpy arrays / floats)."""
    rng = np.random.default_rng(seed)
    p: dict = {"ntypes": NT}
    heavy = np.array([1, 0, 1, 1], bool)           # C, N, O carry pi bonds; H does not
    hh = heavy[:, None] & heavy[None, :]

    # ---- per type
    p["mass"] = MASS.copy()
    p["val"] = np.array([4.0, 1.0, 3.0, 2.0])
    p["vale"] = np.array([4.0, 1.0, 5.0, 6.0])
    p["valboc"] = np.array([4.0, 1.0, 4.0, 4.0])
    p["valang"] = np.array([4.0, 1.0, 4.0, 4.0])
    p["p_lp2"] = np.array([0.0, 0.0, rng.uniform(1, 5), rng.uniform(20, 40)])
    p["p_ovun2"] = rng.uniform(-16, -3, NT)
    p["p_ovun5"] = np.array([rng.uniform(5, 30), rng.uniform(0, 2), rng.uniform(5, 30), rng.uniform(5, 30)])
    p["p_val3"] = rng.uniform(1.0, 4.0, NT)
    p["p_val5"] = rng.uniform(1.0, 3.0, NT)
    p["chi"] = np.array([rng.uniform(120, 170), rng.uniform(80, 120), rng.uniform(150, 190), rng.uniform(180, 220)])
    p["eta"] = rng.uniform(300, 450, NT)
    p["gamma_t"] = rng.uniform(0.5, 1.0, NT)
    p["hb"] = np.array([0, 1, 2, 2], np.int32)

    # ---- per pair (symmetric)
    p["r0s"] = _R0 * _sym(rng, 0.98, 1.02)
    p["r0p"] = np.where(hh, _sym(rng, 1.10, 1.30), 0.0)
    p["r0pp"] = np.where(hh, _sym(rng, 1.00, 1.20), 0.0)
    p["p_bo1"] = _sym(rng, -0.15, -0.07)
    p["p_bo2"] = _sym(rng, 6.0, 9.0)
    p["p_bo3"] = _sym(rng, -0.25, -0.05)
    p["p_bo4"] = _sym(rng, 5.0, 15.0)
    p["p_bo5"] = _sym(rng, -0.25, -0.05)
    p["p_bo6"] = _sym(rng, 10.0, 40.0)
    p["p_boc3"] = _sym(rng, 4.0, 10.0)
    p["p_boc4"] = _sym(rng, 2.0, 8.0)
    p["p_boc5"] = _sym(rng, 0.0, 5.0)
    flags = np.ones((NT, NT))
    flags[1, 1] = 0.0                                # H-H: no f1 and no f4/f5 correction
    p["ovc"] = flags.copy()
    p["v13"] = flags.copy()
    p["De_s"] = _sym(rng, 60.0, 160.0)
    p["De_p"] = np.where(hh, _sym(rng, 50.0, 150.0), 0.0)
    p["De_pp"] = np.where(hh, _sym(rng, 30.0, 100.0), 0.0)
    p["p_be1"] = _sym(rng, -0.5, 0.5)
    p["p_be2"] = _sym(rng, 0.3, 1.2)
    p["p_ovun1"] = _sym(rng, 0.2, 1.0)
    # van der Waals and Coulomb shielding: per type, combined by geometric means
    d_t = rng.uniform(0.05, 0.2, NT)
    rv_t = rng.uniform(1.6, 2.0, NT)
    al_t = rng.uniform(9.0, 11.0, NT)
    gw_t = rng.uniform(1.5, 7.0, NT)
    p["vdw_D"] = np.sqrt(np.outer(d_t, d_t))
    p["vdw_rv"] = 2.0 * np.sqrt(np.outer(rv_t, rv_t))
    p["vdw_alpha"] = np.sqrt(np.outer(al_t, al_t))
    p["vdw_gw"] = np.sqrt(np.outer(gw_t, gw_t))
    p["gamma"] = np.sqrt(np.outer(p["gamma_t"], p["gamma_t"]))

    # ---- per triple (i, j, k), symmetric in i <-> k
    def sym3(lo, hi):
        a = rng.uniform(lo, hi, (NT, NT, NT))
        return 0.5 * (a + a.transpose(2, 1, 0))
    p["th00"] = np.deg2rad(sym3(65.0, 85.0))
    p["p_val1"] = sym3(10.0, 50.0)
    p["p_val2"] = sym3(0.5, 3.0)
    p["p_val4"] = sym3(1.0, 2.0)
    p["p_val7"] = sym3(0.5, 2.0)
    p["p_pen1"] = sym3(0.0, 20.0)
    p["p_coa1"] = sym3(-20.0, 0.0)

    # ---- per torsion centre pair (j, k), symmetric
    p["V1"] = _sym(rng, -5.0, 5.0)
    p["V2"] = _sym(rng, 0.0, 60.0)
    p["V3"] = _sym(rng, -1.0, 1.0)
    p["p_tor1"] = _sym(rng, -8.0, -2.0)
    p["p_cot1"] = _sym(rng, -3.0, 0.0)

    # ---- per H-bond (X, Z)
    p["r0hb"] = rng.uniform(1.8, 2.2, (NT, NT))
    p["p_hb1"] = rng.uniform(-5.0, -1.0, (NT, NT))
    p["p_hb2"] = rng.uniform(1.0, 5.0, (NT, NT))
    p["p_hb3"] = rng.uniform(2.0, 6.0, (NT, NT))

    # ---- general
    gen = dict(p_boc1=(40, 60), p_boc2=(8, 11), p_lp1=(5.5, 7.0), p_ovun3=(20, 60),
               p_ovun4=(0.5, 1.0), p_ovun6=(1.0, 2.0), p_ovun7=(6.0, 12.0), p_ovun8=(10.0, 15.0),
               p_val6=(5.0, 15.0), p_val8=(1.5, 2.5), p_val9=(1.0, 1.1), p_val10=(0.8, 2.0),
               p_pen2=(5.0, 8.0), p_pen3=(0.0, 0.5), p_pen4=(2.0, 4.0), p_coa2=(2.0, 6.0),
               p_coa3=(2.0, 3.0), p_coa4=(0.5, 1.5), p_tor2=(3.0, 6.0), p_tor3=(4.0, 8.0),
               p_tor4=(1.0, 3.0), p_cot2=(1.5, 2.5), p_vdW1=(1.4, 1.7))
    for k in GENERAL:
        if k == "k_e":
            continue
        lo, hi = gen[k]
        p[k] = float(rng.uniform(lo, hi))
    p["k_e"] = 332.06371                              # kcal A / (mol e^2)
    return p


def params_without(p: dict, **zero) -> dict:
    """Copy of p with the named table entries multiplied by 0 (term isolation in tests)."""
    q = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in p.items()}
    for k in zero:
        q[k] = q[k] * 0.0
    return q
