"""Value pins of the oracle's bond-order corrections and energy terms (CPU only).

Each test builds a two- to four-atom molecule in an open box and evaluates the oracle's
Model.energy at a special point: one chosen so that the term under test collapses to a
closed form the mathematics fixes. Examples: a log-sum-exp of equal arguments, a logistic
function at zero, an exponent equal to one, or a count of whole electron pairs. A
dropped factor, a flipped sign or a swapped index in the term would move the oracle off
the closed form. The parameter tables are copies of the seeded set with a few entries
set by hand (documented per test), so the special points are exact.

Forms (Sec. 2.1 lists the terms; the functional forms are the standard ReaxFF forms the
oracle states): f1..f5 bond-order corrections, E_bond, n_lp / E_lp, S / Delta_lpc /
E_over / E_under, SBO / SBO2 / theta0 (through the position of the valence-angle
minimum), f7 / f8, E_pen / f9, E_coa, and the torsion's f10 / f11 / V2 term.
"""
import math

import numpy as np
import pytest
from scipy.optimize import minimize_scalar

import oracle
import synth
from oracle import reaxff_oracle as ro

OPTS = dict(synth.OPTIONS_DEFAULT)
BOX = np.array([30.0, 30.0, 30.0])
C_, H_, N_, O_ = 0, 1, 2, 3


def _copy(P):
    return {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in P.items()}


def _steep(P):
    """Bond orders that vanish beyond ~1.1 r0 (only the intended bonds form)."""
    Q = _copy(P)
    Q["p_bo2"][:] = 20.0
    Q["p_bo4"][:] = 30.0
    Q["p_bo6"][:] = 40.0
    return Q


def _no_corr(P):
    """Corrections off for every pair: BO = BO' (f1 = f4 = f5 = 1)."""
    Q = _copy(P)
    Q["ovc"][:] = 0.0
    Q["v13"][:] = 0.0
    return Q


def _run(P, types, x, mask=None):
    types = np.asarray(types, np.int64)
    m = oracle.Model(P, types, BOX, OPTS)
    L = m.lists(np.asarray(x, float))
    out = m.energy(np.asarray(x, float), np.zeros(len(types)), L, need_grad=False, term_mask=mask)
    return out, L


def _pair(r, t0, t1):
    return [t0, t1], np.array([[15.0, 15.0, 15.0], [15.0 + r, 15.0, 15.0]])


def _raw_bo(P, r, a, b):
    """Uncorrected sigma, pi, pi-pi parts (before the bo_cut shift) of the pair (a, b) at r;
    bo_prime_np is pinned separately by its value at r0."""
    bs, bp, bpp = ro.bo_prime_np(np.array([r]), np.array([a]), np.array([b]), P, OPTS["bo_cut"])
    return float(bs[0]), float(bp[0]), float(bpp[0])


# ======================================================================================
# f1 (over-coordination correction)
# ======================================================================================
def test_f1_is_one_when_both_deltas_vanish(params):
    """Delta'_i = Delta'_j = 0 gives f2 = 2, f3 = -(1/p_boc2) ln 1 = 0, so f1 = 1 exactly.
    Two carbons with Val set to their BO' (Val does not enter BO')."""
    types, x = _pair(1.45, C_, C_)
    out, _ = _run(params, types, x)
    bop = out["parts"]["bo_prime"][0]
    P = _copy(params)
    P["val"][C_] = bop
    out2, _ = _run(P, types, x)
    assert out2["parts"]["bo_prime"][0] == bop
    assert out2["parts"]["f1"][0] == pytest.approx(1.0, abs=2e-15)


@pytest.mark.parametrize("delta", [0.3, -0.2, 0.05])
def test_f1_with_equal_deltas(params, delta):
    """Equal Delta' = d on both ends: f3 is the log of a mean of equal exponentials, so
    f3 = d exactly; f2 = 2 exp(-p_boc1 d); f1 = (Val + f2) / (Val + f2 + d)."""
    types, x = _pair(1.45, C_, C_)
    out, _ = _run(params, types, x)
    bop = out["parts"]["bo_prime"][0]
    P = _copy(params)
    P["p_boc1"] = 2.0
    P["val"][C_] = bop - delta
    f1 = _run(P, types, x)[0]["parts"]["f1"][0]
    V = bop - delta
    f2 = 2.0 * math.exp(-2.0 * delta)
    assert f1 == pytest.approx((V + f2) / (V + f2 + delta), rel=1e-13)


def test_f1_soft_minimum_of_unequal_deltas(params):
    """Unequal Delta' (C: +0.25, O: -0.15) with p_boc1 = 0 (f2 = 2) and p_boc2 = 400: f3 is a
    smooth minimum, f3 = min(Delta') + ln 2 / p_boc2 up to exp(-160); f1 averages the two
    ends' ratios, each with its own Val."""
    types, x = _pair(1.40, C_, O_)
    out, _ = _run(params, types, x)
    bop = out["parts"]["bo_prime"][0]
    P = _copy(params)
    P["p_boc1"] = 0.0
    P["p_boc2"] = 400.0
    d_c, d_o = 0.25, -0.15
    P["val"][C_] = bop - d_c
    P["val"][O_] = bop - d_o
    f1 = _run(P, types, x)[0]["parts"]["f1"][0]
    f3 = min(d_c, d_o) + math.log(2.0) / 400.0
    vc, vo = bop - d_c, bop - d_o
    want = 0.5 * ((vc + 2.0) / (vc + 2.0 + f3) + (vo + 2.0) / (vo + 2.0 + f3))
    assert f1 == pytest.approx(want, rel=1e-13)


# ======================================================================================
# f4, f5 (1-3 bond-order correction) and how the factors enter BO, BOpi, BOpipi
# ======================================================================================
def test_f4_f5_at_their_switching_points(params):
    """f4 = 1 / (1 + exp(-p_boc3 (p_boc4 BO'^2 - Delta'boc_i) + p_boc5)). With Valboc of C set
    so that p_boc4 BO'^2 = Delta'boc_C, f4 = 1 / (1 + e^p_boc5); with Valboc of O set so
    that p_boc4 BO'^2 - Delta'boc_O = p_boc5 / p_boc3, f5 = 1/2 (C is the bond's i end).
    With f1 off: BO = BO' f4 f5, BOpi = BO'pi f4 f5, BOpipi = BO'pipi f4 f5."""
    r = 1.40
    types, x = _pair(r, C_, O_)
    P = _copy(params)
    P["ovc"][:] = 0.0
    out, _ = _run(P, types, x)
    bop = out["parts"]["bo_prime"][0]
    p3, p4, p5 = P["p_boc3"][C_, O_], P["p_boc4"][C_, O_], P["p_boc5"][C_, O_]
    P["valboc"][C_] = bop - p4 * bop * bop
    P["valboc"][O_] = bop - (p4 * bop * bop - p5 / p3)
    pr = _run(P, types, x)[0]["parts"]
    f4, f5 = pr["f4"][0], pr["f5"][0]
    assert f4 == pytest.approx(1.0 / (1.0 + math.exp(p5)), rel=1e-13)
    assert f5 == pytest.approx(0.5, rel=1e-13)
    assert pr["f1"][0] == 1.0
    _, bp, bpp = _raw_bo(P, r, C_, O_)
    fac = 0.5 / (1.0 + math.exp(p5))
    assert pr["bo"][0] == pytest.approx(bop * fac, rel=1e-13)
    assert pr["bo_pi"][0] == pytest.approx(bp * fac, rel=1e-13)
    assert pr["bo_pp"][0] == pytest.approx(bpp * fac, rel=1e-12)


def test_pi_bond_orders_take_f1_squared(params):
    """With f4 = f5 = 1 and Delta' = d on both ends: BO / BO' = f1 while BOpi / BO'pi and
    BOpipi / BO'pipi = f1^2 (f1 from the equal-delta closed form)."""
    d = 0.3
    r = float(params["r0pp"][C_, C_])         # BO'pipi = exp(p_bo5) there
    types, x = _pair(r, C_, C_)
    P = _copy(params)
    P["v13"][:] = 0.0
    out, _ = _run(P, types, x)
    bop = out["parts"]["bo_prime"][0]
    P["p_boc1"] = 2.0
    P["val"][C_] = bop - d
    pr = _run(P, types, x)[0]["parts"]
    V, f2 = bop - d, 2.0 * math.exp(-2.0 * d)
    f1 = (V + f2) / (V + f2 + d)
    _, bp, bpp = _raw_bo(P, r, C_, C_)
    assert bp > 0.1 and bpp > 1e-3
    assert pr["bo"][0] == pytest.approx(bop * f1, rel=1e-13)
    assert pr["bo_pi"][0] == pytest.approx(bp * f1 * f1, rel=1e-13)
    assert pr["bo_pp"][0] == pytest.approx(bpp * f1 * f1, rel=1e-12)


# ======================================================================================
# bond energy
# ======================================================================================
@pytest.mark.parametrize("b", [0.55, 0.9])
def test_bond_energy_sigma_at_a_chosen_bond_order(params, b):
    """Corrections off, pi energies zeroed: BOsig = BO'sig - bo_cut, and the C-C distance is
    chosen by inverting BO'sig(r) so that BOsig = b. Then E_bond = -De_s b exp(p_be1 (1 -
    b^p_be2)) (the scalar form at that bond order)."""
    P = _no_corr(params)
    P["De_p"][:] = 0.0
    P["De_pp"][:] = 0.0
    cut = OPTS["bo_cut"]
    r0, p1, p2 = P["r0s"][C_, C_], P["p_bo1"][C_, C_], P["p_bo2"][C_, C_]
    r = r0 * (math.log((b + cut) / (1.0 + cut)) / p1) ** (1.0 / p2)
    types, x = _pair(r, C_, C_)
    out, _ = _run(P, types, x, mask=("bond",))
    pr = out["parts"]
    assert pr["bo"][0] - pr["bo_pi"][0] - pr["bo_pp"][0] == pytest.approx(b, rel=1e-12)
    De, pb1, pb2 = P["De_s"][C_, C_], P["p_be1"][C_, C_], P["p_be2"][C_, C_]
    assert out["E"]["bond"] == pytest.approx(-De * b * math.exp(pb1 * (1.0 - b ** pb2)), rel=1e-12)


@pytest.mark.parametrize("which", ["pi", "pp"])
def test_bond_energy_pi_parts_at_their_r0(params, which):
    """Corrections off, only one of the pi energies kept: at r = r0pi, BO'pi = exp(p_bo3), so
    E_bond = -De_p exp(p_bo3) (and likewise -De_pp exp(p_bo5) at r = r0pipi)."""
    P = _no_corr(params)
    P["De_s"][:] = 0.0
    if which == "pi":
        P["De_pp"][:] = 0.0
        r, want = P["r0p"][C_, O_], -P["De_p"][C_, O_] * math.exp(P["p_bo3"][C_, O_])
    else:
        P["De_p"][:] = 0.0
        r, want = P["r0pp"][C_, O_], -P["De_pp"][C_, O_] * math.exp(P["p_bo5"][C_, O_])
    types, x = _pair(r, C_, O_)
    out, _ = _run(P, types, x, mask=("bond",))
    assert out["E"]["bond"] == pytest.approx(want, rel=1e-13)


# ======================================================================================
# lone pairs
# ======================================================================================
@pytest.mark.parametrize("k", [0, 1, 2, 3, 4, 5])
def test_lone_pairs_count_whole_electron_pairs(params, k):
    """With k surplus valence electrons (Delta_e = -k): n_lp = floor(k/2) + exp(-lambda u^2),
    u = 1 for odd k (an unpaired electron) and u = 2 for even k; Delta_lp = (Vale - Val)/2
    - n_lp. lambda = p_lp1 = 1 makes the exponentials large enough to pin u. Even k sits
    on the truncation's jump, so Delta_e is put 1e-9 below it."""
    P = _no_corr(params)
    P["p_lp1"] = 1.0
    types, x = _pair(1.40, O_, O_)
    out, _ = _run(P, types, x)
    sbo = out["parts"]["sumbo"][0]
    eps = 1e-9 if k % 2 == 0 else 0.0
    P["vale"][O_] = sbo + k + eps
    pr = _run(P, types, x)[0]["parts"]
    if k % 2:
        want = (k - 1) / 2 + math.exp(-1.0)
    else:
        want = k / 2 + math.exp(-4.0)
    assert pr["nlp"] == pytest.approx([want, want], abs=1e-8)
    nopt = 0.5 * (P["vale"][O_] - P["val"][O_])
    assert pr["dlp"] == pytest.approx([nopt - want] * 2, abs=1e-8)


def test_lone_pair_energy_for_a_missing_and_a_surplus_pair(params):
    """E_lp = p_lp2 Delta_lp / (1 + exp(-75 Delta_lp)): one missing lone pair (Delta_lp = 1
    up to exp(-4 lambda)) costs p_lp2; a surplus pair (Delta_lp = -1) costs nothing (the
    switch gives exp(-75)); Delta_lp = 0 gives 0. lambda = 30 makes exp(-4 lambda) vanish."""
    P = _no_corr(params)
    P["p_lp1"] = 30.0
    types, x = _pair(1.40, O_, O_)
    sbo = _run(P, types, x)[0]["parts"]["sumbo"][0]
    P["vale"][O_] = sbo + 2.0 + 1e-9          # two surplus electrons: n_lp = 1
    lp2 = P["p_lp2"][O_]
    for nopt, want in ((2.0, lp2), (0.0, 0.0), (1.0, 0.0)):
        P["val"][O_] = P["vale"][O_] - 2.0 * nopt
        out = _run(P, types, x, mask=("lp",))[0]
        assert out["parts"]["dlp"] == pytest.approx([nopt - 1.0] * 2, abs=1e-8)
        assert out["E"]["lp"] == pytest.approx(2.0 * want, rel=1e-8, abs=1e-12 * lp2)


# ======================================================================================
# S, Delta_lpc, over- and under-coordination
# ======================================================================================
def _co_setup(params, lam=60.0):
    """C=O pair (pi bonds), corrections off, lambda large: returns (P, types, x, sum BO)."""
    P = _no_corr(params)
    P["p_lp1"] = lam
    types, x = _pair(1.30, C_, O_)
    sbo = _run(P, types, x)[0]["parts"]["sumbo"]
    assert sbo[0] == sbo[1]
    return P, types, x, float(sbo[0])


def test_S_sums_the_neighbours_excess_times_pi_order(params):
    """S_i = sum_j (Delta_j - Delta_lp_j)(BOpi_ij + BOpipi_ij): the carbon is over-coordinated
    by 0.5 with no lone-pair deficit, the oxygen has Delta = Delta_lp = 0; so S_O = 0.5 (BO'pi
    + BO'pipi) and S_C = 0 (each atom sees its neighbour's excess, not its own)."""
    P, types, x, sbo = _co_setup(params)
    P["val"][C_] = sbo - 0.5
    P["vale"][C_] = P["val"][C_]                # n_lp,opt = 0, Delta_e = +0.5: n_lp = 0
    P["val"][O_] = sbo                          # Delta_O = 0
    P["vale"][O_] = sbo + 4.0                   # n_lp = 2 = n_lp,opt
    pr = _run(P, types, x)[0]["parts"]
    _, bp, bpp = _raw_bo(P, 1.30, C_, O_)
    assert pr["dlp"] == pytest.approx([0.0, 0.0], abs=1e-12)
    assert pr["S"][0] == pytest.approx(0.0, abs=1e-14)
    assert pr["S"][1] == pytest.approx(0.5 * (bp + bpp), rel=1e-12)


def test_delta_lpc_divides_the_lone_pair_deficit(params):
    """Delta_lpc = Delta - Delta_lp / (1 + p_ovun3 exp(p_ovun4 S)). O-H (no pi bond: S = 0)
    with Delta_O = 0 and one surplus electron (Delta_lp = 1/2): Delta_lpc = -1/2 / (1 +
    p_ovun3). On C=O with the carbon's excess 0.5 (so S_O = 0.5 (BO'pi + BO'pipi)):
    Delta_lpc,O = -1/2 / (1 + p_ovun3 exp(p_ovun4 S_O))."""
    P = _no_corr(params)
    P["p_lp1"] = 60.0
    types, x = _pair(0.97, O_, H_)
    sbo = _run(P, types, x)[0]["parts"]["sumbo"][0]
    P["val"][O_] = sbo
    P["vale"][O_] = sbo + 1.0
    pr = _run(P, types, x)[0]["parts"]
    assert pr["S"][0] == 0.0
    assert pr["dlp"][0] == pytest.approx(0.5, abs=1e-12)
    assert pr["dlpc"][0] == pytest.approx(-0.5 / (1.0 + P["p_ovun3"]), rel=1e-12)

    P, types, x, sbo = _co_setup(params)
    P["val"][C_] = sbo - 0.5
    P["vale"][C_] = P["val"][C_]
    P["val"][O_] = sbo
    P["vale"][O_] = sbo + 1.0
    pr = _run(P, types, x)[0]["parts"]
    _, bp, bpp = _raw_bo(P, 1.30, C_, O_)
    S = 0.5 * (bp + bpp)
    assert pr["dlpc"][1] == pytest.approx(-0.5 / (1.0 + P["p_ovun3"] * math.exp(P["p_ovun4"] * S)), rel=1e-12)
    assert pr["dlpc"][0] == pytest.approx(0.5, abs=1e-12)      # no lone-pair deficit: Delta


def _cc_over(params, delta, **over):
    """C-C with Delta = delta on both atoms and no lone pairs (Delta_lpc = delta)."""
    P = _no_corr(params)
    P["p_lp1"] = 60.0
    for k, v in over.items():
        P[k] = v
    types, x = _pair(1.45, C_, C_)
    sbo = _run(P, types, x)[0]["parts"]["sumbo"][0]
    P["val"][C_] = sbo - delta
    P["vale"][C_] = P["val"][C_]
    return P, types, x, sbo


def test_over_and_under_vanish_at_zero_delta_lpc(params):
    P, types, x, _ = _cc_over(params, 0.0)
    out = _run(P, types, x, mask=("over", "under"))[0]
    assert out["parts"]["dlpc"] == pytest.approx([0.0, 0.0], abs=1e-12)
    assert abs(out["E"]["over"]) < 1e-10 and abs(out["E"]["under"]) < 1e-10


def test_over_coordination_closed_forms(params):
    """E_over = [sum_j p_ovun1 De_s BO] Delta_lpc / (Delta_lpc + Val) / (1 + exp(p_ovun2
    Delta_lpc)). With p_ovun2 = 0 and Delta_lpc = Val (over-coordinated by Val): each atom
    gives 1/4 p_ovun1 De_s BO. With p_ovun2 back, the ratio is 2 / (1 + exp(p_ovun2 Val))."""
    P0 = _copy(params)
    P0["p_ovun2"] = P0["p_ovun2"] * 0.0
    types, x = _pair(1.45, C_, C_)
    sbo = _run(_no_corr(P0), types, x)[0]["parts"]["sumbo"][0]
    P, types, x, _ = _cc_over(P0, sbo / 2.0)             # Delta = Val = sum BO / 2
    out = _run(P, types, x, mask=("over",))[0]
    assert out["parts"]["dlpc"] == pytest.approx([sbo / 2] * 2, rel=1e-12)
    base = 2.0 * 0.25 * P["p_ovun1"][C_, C_] * P["De_s"][C_, C_] * sbo
    assert out["E"]["over"] == pytest.approx(base, rel=1e-7)          # the 1e-8 guard term
    P2, _, _, _ = _cc_over(params, sbo / 2.0)
    e2 = _run(P2, types, x, mask=("over",))[0]["E"]["over"]
    assert e2 / out["E"]["over"] == pytest.approx(2.0 / (1.0 + math.exp(params["p_ovun2"][C_] * sbo / 2)), rel=1e-12)


def test_under_coordination_closed_forms(params):
    """E_under = -p_ovun5 (1 - exp(p_ovun6 Delta_lpc)) / (1 + exp(-p_ovun2 Delta_lpc)) / (1 +
    p_ovun7 exp(p_ovun8 S)). With p_ovun2 = 0, p_ovun7 = 0 and Delta_lpc = -ln 2 / p_ovun6:
    each atom gives -p_ovun5 / 4. With p_ovun7 = 1 and S set by the pi bonds, the last factor
    is 1 / (1 + exp(p_ovun8 S)), S = Delta (BO'pi + BO'pipi)."""
    p6 = params["p_ovun6"]
    d = -math.log(2.0) / p6
    pz = np.zeros_like(params["p_ovun2"])
    P, types, x, _ = _cc_over(params, d, p_ovun2=pz, p_ovun7=0.0)
    out = _run(P, types, x, mask=("under",))[0]
    assert out["parts"]["dlpc"] == pytest.approx([d, d], rel=1e-12)
    assert out["E"]["under"] == pytest.approx(2.0 * -P["p_ovun5"][C_] / 4.0, rel=1e-12)
    P1, _, _, _ = _cc_over(params, d, p_ovun2=pz, p_ovun7=1.0)
    pr = _run(P1, types, x, mask=("under",))[0]
    _, bp, bpp = _raw_bo(P1, 1.45, C_, C_)
    S = d * (bp + bpp)
    assert pr["parts"]["S"] == pytest.approx([S, S], rel=1e-12)
    assert pr["E"]["under"] == pytest.approx(out["E"]["under"] / (1.0 + math.exp(P1["p_ovun8"] * S)), rel=1e-12)
    # the logistic in Delta_lpc: with p_ovun2 back the ratio is 2 / (1 + exp(-p_ovun2 Delta_lpc))
    P2, _, _, _ = _cc_over(params, d, p_ovun7=0.0)
    e2 = _run(P2, types, x, mask=("under",))[0]["E"]["under"]
    assert e2 / out["E"]["under"] == pytest.approx(2.0 / (1.0 + math.exp(-params["p_ovun2"][C_] * d)), rel=1e-12)


# ======================================================================================
# valence angle: SBO, SBO2 and theta0 through the position of the E_val minimum
# ======================================================================================
def _bent(th, t_end, t_mid, b1, b2, t_end2=None):
    """Three atoms end-centre-end: centre at the origin (+15), bond lengths b1, b2, angle th."""
    j = np.array([15.0, 15.0, 15.0])
    i = j + b1 * np.array([math.cos(th), math.sin(th), 0.0])
    k = j + np.array([b2, 0.0, 0.0])
    return [t_end, t_mid, t_end if t_end2 is None else t_end2], np.stack([i, j, k])


def _val_energy(P, types, x):
    return _run(P, types, x, mask=("val",))[0]["E"]["val"]


def _argmin_theta(P, t_end, t_mid, b):
    f = lambda th: _val_energy(P, *_bent(th, t_end, t_mid, b, b))      # noqa: E731
    res = minimize_scalar(f, bounds=(np.deg2rad(80.0), np.deg2rad(175.0)), method="bounded",
                          options=dict(xatol=1e-11))
    return res.x


def _hoh(params, **over):
    """H-O-H with steep bond orders, corrections off, O-H bonds at r0sig: returns (P, b,
    sum BO of O, BO of one O-H bond)."""
    P = _no_corr(_steep(params))
    for k, v in over.items():
        P[k] = v
    b = float(P["r0s"][O_, H_])
    types, x = _bent(np.deg2rad(104.0), H_, O_, b, b)
    pr = _run(P, types, x)[0]["parts"]
    assert len(pr["bo"]) == 2
    return P, b, float(pr["sumbo"][1]), float(pr["bo"][0])


def test_theta0_when_sbo2_is_zero(params):
    """No pi bond and p_val8 = 0: SBO = (1 - prod exp(-BO^8)) (-Delta_angle) < 0 for
    Delta_angle = 0.5, so SBO2 = 0 and theta0 = pi - theta00 (1 - exp(-2 p_val10)); the
    valence-angle energy is smallest there."""
    P, b, sbo, _ = _hoh(params, p_val8=0.0)
    P["valang"][O_] = sbo - 0.5
    th0 = math.pi - P["th00"][H_, O_, H_] * (1.0 - math.exp(-2.0 * P["p_val10"]))
    assert _argmin_theta(P, H_, O_, b) == pytest.approx(th0, abs=1e-6)


def test_theta0_is_linear_when_sbo2_is_two(params):
    """SBO >= 2 gives SBO2 = 2 and theta0 = pi: E_val vanishes exactly at the linear
    geometry and grows as the angle closes."""
    P, b, sbo, bo = _hoh(params, p_val8=0.0)
    assert 20.0 * (1.0 - math.exp(-2.0 * bo ** 8)) > 2.0
    P["valang"][O_] = sbo + 20.0
    e = [_val_energy(P, *_bent(np.deg2rad(a), H_, O_, b, b)) for a in (180.0, 175.0, 160.0)]
    assert e[0] == 0.0
    assert 0.0 < e[1] < e[2]


def test_theta0_with_sbo_between_one_and_two(params):
    """p_val9 = 1 makes SBO2 = SBO on [0, 2]. Delta_angle set so that SBO = 1.3 (no pi bond,
    p_val8 = 0): theta0 = pi - theta00 (1 - exp(-0.7 p_val10))."""
    P, b, sbo, bo = _hoh(params, p_val8=0.0, p_val9=1.0)
    P["valang"][O_] = sbo + 1.3 / (1.0 - math.exp(-2.0 * bo ** 8))
    th0 = math.pi - P["th00"][H_, O_, H_] * (1.0 - math.exp(-0.7 * P["p_val10"]))
    assert _argmin_theta(P, H_, O_, b) == pytest.approx(th0, abs=1e-6)


def test_sbo_counts_the_lone_pairs_with_p_val8(params):
    """SBO = sum(BOpi + BOpipi) + (1 - prod exp(-BO^8)) (-Delta_angle - p_val8 n_lp): with the
    oxygen's n_lp (pinned above) and Delta_angle = -(p_val8 n_lp + 1.3 / (1 - prod)), SBO =
    1.3 again and the minimum sits at the same theta0."""
    P, b, sbo, bo = _hoh(params, p_val9=1.0)
    types, x = _bent(np.deg2rad(104.0), H_, O_, b, b)
    nlp = float(_run(P, types, x)[0]["parts"]["nlp"][1])
    assert nlp == pytest.approx(2.0, abs=1e-3)
    P["valang"][O_] = sbo + P["p_val8"] * nlp + 1.3 / (1.0 - math.exp(-2.0 * bo ** 8))
    th0 = math.pi - P["th00"][H_, O_, H_] * (1.0 - math.exp(-0.7 * P["p_val10"]))
    assert _argmin_theta(P, H_, O_, b) == pytest.approx(th0, abs=1e-6)


def test_sbo_sums_the_pi_bond_orders(params):
    """C-C-H centred on the first C, the C-C bond at r0pipi (both pi parts large), the C-H
    bond without pi, Delta_angle = 0, p_val9 = 1: SBO = BO'pi + BO'pipi of the C-C bond
    (< 2), theta0 = pi - theta00 (1 - exp(-p_val10 (2 - SBO)))."""
    P = _no_corr(_steep(params))
    P["p_val9"] = 1.0
    b1, b2 = float(P["r0pp"][C_, C_]), float(P["r0s"][C_, H_])
    types, x = _bent(np.deg2rad(115.0), C_, C_, b1, b2, t_end2=H_)
    pr = _run(P, types, x)[0]["parts"]
    assert len(pr["bo"]) == 2
    P["valang"][C_] = float(pr["sumbo"][1])
    _, bp, bpp = _raw_bo(P, b1, C_, C_)
    sbo = bp + bpp
    assert 1.0 < sbo < 2.0 and bpp > 0.3
    th0 = math.pi - P["th00"][C_, C_, H_] * (1.0 - math.exp(-P["p_val10"] * (2.0 - sbo)))
    f = lambda th: _val_energy(P, *_bent(th, C_, C_, b1, b2, t_end2=H_))      # noqa: E731
    res = minimize_scalar(f, bounds=(np.deg2rad(80.0), np.deg2rad(179.9)), method="bounded",
                          options=dict(xatol=1e-11))
    assert res.x == pytest.approx(th0, abs=1e-6)


@pytest.mark.parametrize("edge", [1.0, 2.0])
def test_sbo2_is_continuous_at_its_branch_points(params, edge):
    """SBO2 changes form at SBO = 1 and 2 (SBO^p9, 2 - (2 - SBO)^p9, 2); with p_val9 = 1.07
    E_val at a fixed angle is continuous across each edge (a wrong branch jumps)."""
    P, b, sbo, bo = _hoh(params, p_val8=0.0, p_val9=1.07)
    denom = 1.0 - math.exp(-2.0 * bo ** 8)
    x3 = _bent(np.deg2rad(120.0), H_, O_, b, b)
    es = []
    for s in (edge - 1e-7, edge + 1e-7):
        P["valang"][O_] = sbo + s / denom
        es.append(_val_energy(P, *x3))
    assert abs(es[1] - es[0]) < 1e-5 * abs(es[0])


# ======================================================================================
# valence angle: f7 and f8
# ======================================================================================
def _hoh_flat(params, **over):
    """H-O-H at 90 deg with theta0 = pi (p_val10 = 0) and p_val2 = 30: the angle factor
    1 - exp(-30 (pi/2)^2) is 1 to 1e-32, so E_val = p_val1 f7(BO)^2 f8(Delta_angle)."""
    P, b, sbo, bo = _hoh(params, p_val10=0.0, **over)
    P["p_val2"][:] = 30.0
    return P, _bent(np.pi / 2, H_, O_, b, b), sbo, bo


@pytest.mark.parametrize("p4", [1.0, 2.0])
def test_f7_at_zero_delta_angle(params, p4):
    """Delta_angle = 0 makes f8 = p5 - (p5 - 1) 3/3 = 1; then E_val = p_val1 (1 - exp(-p_val3
    BO^p_val4))^2 for the two equal O-H bonds."""
    P, geom, sbo, bo = _hoh_flat(params)
    P["valang"][O_] = sbo
    P["p_val4"][:] = p4
    f7 = 1.0 - math.exp(-P["p_val3"][O_] * bo ** p4)
    assert _val_energy(P, *geom) == pytest.approx(P["p_val1"][H_, O_, H_] * f7 * f7, rel=1e-12)


def test_f8_limits(params):
    """f8 = p5 - (p5 - 1)(2 + e^(p6 D)) / (1 + e^(p6 D) + e^(-p7 D)), D = Delta_angle: an
    under-coordinated centre (D = -0.5, p_val7 = 60) scales E_val by p_val5; an
    over-coordinated one (D = +0.5, p_val6 = 60) leaves it at f8 = 1."""
    P, geom, sbo, _ = _hoh_flat(params)
    P["valang"][O_] = sbo
    e0 = _val_energy(P, *geom)
    P["p_val7"][:] = 60.0
    P["valang"][O_] = sbo + 0.5
    assert _val_energy(P, *geom) / e0 == pytest.approx(P["p_val5"][O_], rel=1e-10)
    P["p_val6"] = 60.0
    P["valang"][O_] = sbo - 0.5
    assert _val_energy(P, *geom) / e0 == pytest.approx(1.0, rel=1e-10)


# ======================================================================================
# penalty and coalition
# ======================================================================================
def test_penalty_closed_forms(params):
    """E_pen = p_pen1 f9(Delta_j) exp(-p_pen2 (BO_ij - 2)^2) exp(-p_pen2 (BO_jk - 2)^2),
    f9 = (2 + e^(-p3 D)) / (1 + e^(-p3 D) + e^(p4 D)). p_pen2 = 0 and Delta_O = 0: E_pen =
    p_pen1. p_pen3 = 0 and Delta_O = ln 2 / p_pen4: f9 = 3/4. p_pen2 back: the factor
    exp(-2 p_pen2 (BO - 2)^2) for the two equal bonds."""
    P, b, sbo, bo = _hoh(params)
    geom = _bent(np.deg2rad(104.0), H_, O_, b, b)
    p1 = P["p_pen1"][H_, O_, H_]
    p2 = P["p_pen2"]
    P["p_pen2"] = 0.0
    P["val"][O_] = sbo
    pen = lambda: _run(P, *geom, mask=("pen",))[0]["E"]["pen"]     # noqa: E731
    assert pen() == pytest.approx(p1, rel=1e-13)
    p3 = P["p_pen3"]
    P["p_pen3"] = 0.0
    P["val"][O_] = sbo - math.log(2.0) / P["p_pen4"]
    assert pen() == pytest.approx(0.75 * p1, rel=1e-13)
    P["p_pen3"] = p3
    P["val"][O_] = sbo
    P["p_pen2"] = p2
    assert pen() == pytest.approx(p1 * math.exp(-2.0 * p2 * (bo - 2.0) ** 2), rel=1e-12)


def test_coalition_uses_each_end_atoms_other_bonds(params):
    """Chain H(m)-O(i)-C(j)-H(k): two angles, centred on O and on C. E_coa = p_coa1 / (1 +
    exp(p_coa2 Delta_angle)) exp(-p_coa3 (sumBO_end1 - BO_1)^2) exp(-p_coa3 (sumBO_end2 -
    BO_2)^2) times the p_coa4 factors. With p_coa4 = 0 and Delta_angle = 0 at both centres,
    the O-centred angle sees the C end's other bond (C-H) and the C-centred one the O end's
    other bond (O-H): E_coa = 1/2 p_coa1[H,O,C] exp(-p3 BO_CH^2) + 1/2 p_coa1[O,C,H]
    exp(-p3 BO_OH^2). p_coa2 and p_coa4 are then switched back on one at a time."""
    P = _no_corr(_steep(params))
    b_oh, b_oc, b_ch = (float(P["r0s"][a, c]) for a, c in ((O_, H_), (O_, C_), (C_, H_)))
    o = np.array([15.0, 15.0, 15.0])
    c = o + np.array([b_oc, 0.0, 0.0])
    m = o + b_oh * np.array([math.cos(np.deg2rad(105.0)), math.sin(np.deg2rad(105.0)), 0.0])
    k = c + b_ch * np.array([-math.cos(np.deg2rad(110.0)), -math.sin(np.deg2rad(110.0)), 0.0])
    types, x = [H_, O_, C_, H_], np.stack([m, o, c, k])
    out = _run(P, types, x)[0]
    pr = out["parts"]
    assert len(pr["bo"]) == 3 and out["parts"]["n_angles"] == 2
    bo = {}
    for name, (a, cc, r) in dict(oh=(O_, H_, b_oh), oc=(O_, C_, b_oc), ch=(C_, H_, b_ch)).items():
        bs, bp, bpp = _raw_bo(P, r, a, cc)
        bo[name] = bs + bp + bpp - OPTS["bo_cut"]
    P["valang"][O_] = bo["oh"] + bo["oc"]
    P["valang"][C_] = bo["oc"] + bo["ch"]
    P["p_coa4"] = 0.0
    p3 = P["p_coa3"]
    a1, a2 = P["p_coa1"][H_, O_, C_], P["p_coa1"][O_, C_, H_]
    coa = lambda: _run(P, types, x, mask=("coa",))[0]["E"]["coa"]     # noqa: E731
    want = 0.5 * a1 * math.exp(-p3 * bo["ch"] ** 2) + 0.5 * a2 * math.exp(-p3 * bo["oh"] ** 2)
    assert coa() == pytest.approx(want, rel=1e-12)
    # Delta_angle = -0.3 at the carbon: its angle's switch becomes 1 / (1 + exp(-0.3 p_coa2))
    P["valang"][C_] += 0.3
    want2 = 0.5 * a1 * math.exp(-p3 * bo["ch"] ** 2) + \
        a2 / (1.0 + math.exp(-0.3 * P["p_coa2"])) * math.exp(-p3 * bo["oh"] ** 2)
    assert coa() == pytest.approx(want2, rel=1e-12)
    P["valang"][C_] -= 0.3
    P["p_coa4"] = params["p_coa4"]
    p4 = P["p_coa4"]
    want3 = 0.5 * a1 * math.exp(-p3 * bo["ch"] ** 2) * math.exp(-p4 * ((bo["oh"] - 1.5) ** 2 + (bo["oc"] - 1.5) ** 2)) \
        + 0.5 * a2 * math.exp(-p3 * bo["oh"] ** 2) * math.exp(-p4 * ((bo["oc"] - 1.5) ** 2 + (bo["ch"] - 1.5) ** 2))
    assert coa() == pytest.approx(want3, rel=1e-12)


# ======================================================================================
# torsion: f10, f11 and the V2 term; conjugation amplitude
# ======================================================================================
def _chain(theta, omega, b_end, b_mid):
    """i-j-k-l: end bonds b_end, central bond b_mid, both bond angles theta, dihedral omega."""
    j = np.zeros(3)
    k = np.array([b_mid, 0.0, 0.0])
    i = b_end * np.array([math.cos(theta), math.sin(theta), 0.0])
    l_ = k + b_end * np.array([-math.cos(theta), math.sin(theta) * math.cos(omega), math.sin(theta) * math.sin(omega)])
    return np.stack([i, j, k, l_]) + 15.0


def _tors_setup(params, **over):
    """C4 chain, steep bond orders, corrections off, central bond at r0pi (BO'pi = exp(p_bo3)),
    end bonds at r0sig; only the V2 amplitude; Delta_angle = 0 at j and k (f11 = 1);
    p_tor2 = 60 (f10 = 1 to 1e-20). Returns (P, theta, bond orders (ij, jk, kl), BOpi_jk)."""
    P = _no_corr(_steep(params))
    P["V1"][:] = 0.0
    P["V3"][:] = 0.0
    P["V2"][:] = 2.5
    P["p_tor2"] = 60.0
    for k, v in over.items():
        P[k] = v
    b_end, b_mid = float(P["r0s"][C_, C_]), float(P["r0p"][C_, C_])
    th = np.deg2rad(112.0)
    x = _chain(th, np.pi / 2, b_end, b_mid)
    out = _run(P, np.zeros(4, np.int64), x)[0]
    assert len(out["parts"]["bo"]) == 3 and out["parts"]["n_torsions"] == 1
    bo = []
    for r in (b_end, b_mid, b_end):
        bs, bp, bpp = _raw_bo(P, r, C_, C_)
        bo.append(bs + bp + bpp - OPTS["bo_cut"])
    P["valang"][C_] = bo[0] + bo[1]
    return P, th, (b_end, b_mid), bo, _raw_bo(P, b_mid, C_, C_)[1]


def _tors(P, th, bl, omega, term="tors"):
    x = _chain(th, omega, *bl)
    return _run(P, np.zeros(4, np.int64), x, mask=(term,))[0]["E"][term]


def test_torsion_v2_term_closed_form(params):
    """E_tors = f10 sin th1 sin th2 [... + 1/2 V2 exp(p_tor1 (2 - BOpi_jk - f11)^2)(1 - cos 2w)
    + ...]. With f10 = f11 = 1: at w = 90 deg, E = sin^2 th V2 exp(p_tor1 (1 - BOpi)^2);
    w = 45 deg gives half of that; w = 0 gives 0."""
    P, th, bl, bo, bpi = _tors_setup(params)
    want = math.sin(th) ** 2 * 2.5 * math.exp(P["p_tor1"][C_, C_] * (1.0 - bpi) ** 2)
    e90 = _tors(P, th, bl, np.pi / 2)
    assert e90 == pytest.approx(want, rel=1e-11)
    assert _tors(P, th, bl, np.pi / 4) == pytest.approx(0.5 * e90, rel=1e-10)
    assert abs(_tors(P, th, bl, 0.0)) < 1e-12 * abs(e90)


def test_torsion_f11_and_f10(params):
    """f11 = (2 + e^(-p3 D)) / (1 + e^(-p3 D) + e^(p4 D)), D = Delta_angle_j + Delta_angle_k:
    with p_tor3 = 0 and D = ln 2 / p_tor4, f11 = 3/4. f10 = prod over the three bonds of
    (1 - exp(-p_tor2 BO)): with p_tor2 = 1 the energy is scaled by that product."""
    P, th, bl, bo, bpi = _tors_setup(params, p_tor3=0.0)
    e1 = _tors(P, th, bl, np.pi / 2)
    P["valang"][C_] -= math.log(2.0) / (2.0 * P["p_tor4"])
    e2 = _tors(P, th, bl, np.pi / 2)
    pt1 = P["p_tor1"][C_, C_]
    assert e2 / e1 == pytest.approx(math.exp(pt1 * (1.25 - bpi) ** 2 - pt1 * (1.0 - bpi) ** 2), rel=1e-11)
    P["valang"][C_] += math.log(2.0) / (2.0 * P["p_tor4"])
    P["p_tor2"] = 1.0
    f10 = np.prod([1.0 - math.exp(-b) for b in bo])
    assert _tors(P, th, bl, np.pi / 2) / e1 == pytest.approx(f10, rel=1e-11)


def test_conjugation_amplitude(params):
    """E_conj = p_cot1 prod exp(-p_cot2 (BO - 1.5)^2) [1 + (cos^2 w - 1) sin th1 sin th2]: with
    p_cot2 = 0 and w = 0 the bracket is 1 and E_conj = p_cot1; with p_cot2 back it is scaled
    by the product over the three bonds."""
    P, th, bl, bo, _ = _tors_setup(params)
    P["p_cot1"][:] = -1.7
    pc2 = P["p_cot2"]
    P["p_cot2"] = 0.0
    assert _tors(P, th, bl, 0.0, "conj") == pytest.approx(-1.7, rel=1e-13)
    P["p_cot2"] = pc2
    want = -1.7 * np.prod([math.exp(-pc2 * (b - 1.5) ** 2) for b in bo])
    assert _tors(P, th, bl, 0.0, "conj") == pytest.approx(want, rel=1e-12)
