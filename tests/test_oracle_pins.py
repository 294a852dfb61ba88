"""Pins of the FP64 CPU oracle against what mathematics and the method fix (CPU only).

Each test checks the oracle against something other than itself: exact rational
algebra, brute force, finite differences, invariances, closed forms of special cases
and a dense factorisation.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from oracle import reaxff_oracle as ro
from synth.params import params_without


def _model(P, w):
    return oracle.Model(P, w["types"], w["box"], w["options"])


def _steep(P):
    """Parameter variant whose bond orders vanish beyond ~1.1 r0 (isolates bonds)."""
    Q = params_without(P)
    Q["p_bo2"] = Q["p_bo2"] * 0 + 20.0
    Q["p_bo4"] = Q["p_bo4"] * 0 + 30.0
    Q["p_bo6"] = Q["p_bo6"] * 0 + 40.0
    return Q


# ------------------------------------------------------------------ taper
def test_taper_is_the_unique_degree7_polynomial():
    """Solve Tap(0)=1, Tap'(0)=Tap''(0)=Tap'''(0)=0, Tap(1)=Tap'(1)=Tap''(1)=Tap'''(1)=0 in
    exact rationals and compare with the oracle's coefficients."""
    rows, rhs = [], []
    for x0, val in ((0, 1), (1, 0)):
        for d in range(4):
            row = []
            for k in range(8):
                if k < d:
                    row.append(Fraction(0))
                else:
                    c = Fraction(1)
                    for m in range(d):
                        c *= (k - m)
                    row.append(c * (Fraction(x0) ** (k - d) if k - d > 0 else Fraction(1)))
            rows.append(row)
            rhs.append(Fraction(val if d == 0 else 0))
    n = 8
    A = [r + [b] for r, b in zip(rows, rhs)]
    for c in range(n):
        p = next(r for r in range(c, n) if A[r][c] != 0)
        A[c], A[p] = A[p], A[c]
        for r in range(n):
            if r != c and A[r][c] != 0:
                f = A[r][c] / A[c][c]
                A[r] = [a - f * b for a, b in zip(A[r], A[c])]
    coef = [A[k][n] / A[k][k] for k in range(n)]
    assert [float(c) for c in coef] == list(ro.TAPER_COEF)
    assert ro.taper(0.0, 10.0) == 1.0
    assert abs(ro.taper(10.0, 10.0)) < 1e-12


# ------------------------------------------------------------------ lists
@pytest.mark.parametrize("name", ["petn464", "cluster300"])
def test_cell_list_equals_brute_force(name):
    w = synth.workload(name)
    a = oracle.far_list_bruteforce(w["x"], w["box"], 10.0)
    b = oracle.far_list_cells(w["x"], w["box"], 10.0)
    n = len(w["x"])
    ka = np.sort(oracle.sort_key(*a, n))
    kb = np.sort(oracle.sort_key(*b, n))
    assert len(np.unique(ka)) == len(ka)
    assert np.array_equal(ka, kb)


def test_cell_list_three_cells_per_axis():
    types, x, box = synth.random_cluster(700, (31.0, 22.0, 20.5), seed=3)
    a = oracle.far_list_bruteforce(x, box, 10.0)
    b = oracle.far_list_cells(x, box, 10.0)
    assert np.array_equal(np.sort(oracle.sort_key(*a, 700)), np.sort(oracle.sort_key(*b, 700)))


def test_far_list_plain_loops_tiny():
    """Plain-Python loops over |s| <= 2 images agree with the vectorised brute force
    (shows |s| <= 1 is complete when every box length exceeds the cutoff)."""
    rng = np.random.default_rng(5)
    box = np.array([11.0, 12.5, 10.5])
    x = rng.uniform(0, 1, (14, 3)) * box
    ref = set()
    for i in range(14):
        for j in range(14):
            for sx in range(-2, 3):
                for sy in range(-2, 3):
                    for sz in range(-2, 3):
                        if i == j and sx == sy == sz == 0:
                            continue
                        d = [(x[j][c] - x[i][c]) + s * box[c] for c, s in enumerate((sx, sy, sz))]
                        if (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2] < 100.0:
                            ref.add((i, j, sx, sy, sz))
    i, j, s = oracle.far_list_bruteforce(x, box, 10.0)
    got = {(a, b, *map(int, c)) for a, b, c in zip(i, j, s)}
    assert got == ref


@pytest.mark.parametrize("name", ["petn464", "cluster300"])
def test_no_ambiguous_list_decisions(params, name):
    """No pair sits within 1e-12 (relative) of a list threshold: r^2 vs R^2 and BO' vs bo_cut."""
    w = synth.workload(name)
    o = w["options"]
    i, j, s = oracle.far_list_bruteforce(w["x"], w["box"], 10.5)
    r2 = ro._r2(w["x"], w["box"], i, j, s)
    for R in (o["r_nb"], o["r_bond"], o["r_hb"]):
        assert not np.any(np.abs(r2 - R * R) < 1e-12 * R * R)
    m = r2 < o["r_bond"] ** 2
    bs, bp, bpp = ro.bo_prime_np(np.sqrt(r2[m]), w["types"][i[m]], w["types"][j[m]], params, o["bo_cut"])
    assert not np.any(np.abs(bs + bp + bpp - o["bo_cut"]) < 1e-12 * o["bo_cut"])


# ------------------------------------------------------------------ bond orders
def test_bo_prime_closed_form_at_r0(params):
    P = params
    bo_cut = 1e-3
    for a in range(4):
        for b in range(4):
            bs, _, _ = ro.bo_prime_np(np.array([P["r0s"][a, b]]), np.array([a]), np.array([b]), P, bo_cut)
            assert bs[0] == pytest.approx((1 + bo_cut) * np.exp(P["p_bo1"][a, b]), rel=1e-15)


def test_corrections_off_reduce_to_uncorrected(params):
    P = params_without(params, ovc=1, v13=1)
    w = synth.workload("cluster300")
    m = _model(P, w)
    L = m.lists(w["x"])
    out = m.energy(w["x"], np.zeros(len(w["x"])), L, need_grad=False)
    pr = out["parts"]
    assert np.array_equal(pr["f1"], np.ones_like(pr["f1"]))
    assert np.allclose(pr["bo"], pr["bo_prime"], rtol=0, atol=0)


# ------------------------------------------------------------------ invariances
def _full(P, w, x=None, q=None):
    m = _model(P, w)
    return m.forces(w["x"] if x is None else x, q=q, tol=1e-12)


@pytest.fixture(scope="module")
def cluster_ref(params):
    w = synth.workload("cluster300")
    return w, _full(params, w)


def test_permutation_invariance(params, cluster_ref):
    w, ref = cluster_ref
    perm = np.random.default_rng(1).permutation(len(w["x"]))
    w2 = dict(w, types=w["types"][perm], x=w["x"][perm])
    out = _full(params, w2, q=ref["qeq"]["q"][perm])
    for k in oracle.TERMS:
        assert out["E"][k] == pytest.approx(ref["E"][k], rel=1e-10, abs=1e-9)
    assert np.allclose(out["F"], ref["F"][perm], rtol=1e-9, atol=1e-8)


def test_translation_invariance(params, cluster_ref):
    w, ref = cluster_ref
    x = np.mod(w["x"] + np.array([3.3, -7.1, 11.9]), w["box"])
    out = _full(params, w, x=x, q=ref["qeq"]["q"])
    assert out["E_total"] == pytest.approx(ref["E_total"], rel=1e-11)
    assert np.allclose(out["F"], ref["F"], rtol=1e-8, atol=1e-8)


def test_rotation_invariance_and_zero_torque(params):
    """Open cluster (box far larger than the cluster + cutoff): E is rotation invariant,
    forces rotate with it, net force and torque vanish."""
    t, x, _ = synth.random_cluster(60, (9.0, 9.0, 9.0), seed=11, dmin=1.0)
    box = np.array([60.0, 60.0, 60.0])
    x = x + 25.0
    w = dict(types=t, x=x, box=box, options=dict(synth.OPTIONS_DEFAULT))
    a = _full(params, w)
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
    R = R @ np.array([[1, 0, 0], [0, np.cos(0.4), -np.sin(0.4)], [0, np.sin(0.4), np.cos(0.4)]])
    c = x.mean(0)
    xr = (x - c) @ R.T + c
    b = _full(params, dict(w, x=xr))
    assert b["E_total"] == pytest.approx(a["E_total"], rel=1e-11)
    assert np.allclose(b["F"], a["F"] @ R.T, atol=1e-8 * np.abs(a["F"]).max())
    assert np.abs(a["F"].sum(0)).max() < 1e-9 * np.abs(a["F"]).max()
    torque = np.cross(x - c, a["F"]).sum(0)
    assert np.abs(torque).max() < 1e-8 * np.abs(a["F"]).max() * 10.0


def test_net_force_zero_periodic(params, cluster_ref):
    _, ref = cluster_ref
    assert np.abs(ref["F"].sum(0)).max() < 1e-9 * np.abs(ref["F"]).max()


# ------------------------------------------------------------------ finite differences
@pytest.mark.parametrize("name", ["cluster300", "petn464"])
def test_forces_central_differences(params, name):
    w = synth.workload(name)
    m = _model(params, w)
    out = m.forces(w["x"], tol=1e-12)
    L, q = out["lists"], out["qeq"]["q"]
    rng = np.random.default_rng(2)
    h = 1e-5
    for a in rng.choice(len(w["x"]), 3, replace=False):
        for c in range(3):
            xp, xm = w["x"].copy(), w["x"].copy()
            xp[a, c] += h
            xm[a, c] -= h
            fd = -(m.energy(xp, q, L, need_grad=False)["E_total"] - m.energy(xm, q, L, need_grad=False)["E_total"]) / (2 * h)
            assert out["F"][a, c] == pytest.approx(fd, rel=2e-6, abs=2e-5)


def test_forces_equal_total_derivative_with_requilibrated_charges(params):
    """dE/dq_i = mu at the QEq solution and sum dq = 0, so FD of E with QEq re-solved at
    each displaced geometry equals the fixed-charge force (pins H against E_coul)."""
    w = synth.workload("cluster300")
    m = _model(params, w)
    out = m.forces(w["x"], tol=1e-13)
    L = out["lists"]
    h = 1e-5
    for a, c in ((7, 0), (123, 2)):
        es = []
        for sgn in (1, -1):
            x = w["x"].copy()
            x[a, c] += sgn * h
            q = m.qeq(x, L, tol=1e-13)["q"]
            es.append(m.energy(x, q, L, need_grad=False)["E_total"])
        fd = -(es[0] - es[1]) / (2 * h)
        assert out["F"][a, c] == pytest.approx(fd, rel=1e-6, abs=1e-5)


def test_virial_diagonal_strain_fd(params):
    """-dE/d(eps_aa) under a homogeneous scaling of positions and box (fixed q) equals the
    virial's diagonal; the virial is symmetric."""
    w = synth.workload("cluster300")
    m = _model(params, w)
    out = m.forces(w["x"], tol=1e-12)
    L, q, W = out["lists"], out["qeq"]["q"], out["W"]
    assert np.allclose(W, W.T, rtol=1e-9, atol=1e-7 * np.abs(W).max())
    h = 1e-6
    for a in range(3):
        es = []
        for sgn in (1, -1):
            s = np.ones(3)
            s[a] += sgn * h
            mm = oracle.Model(params, w["types"], w["box"] * s, w["options"])
            es.append(mm.energy(w["x"] * s, q, L, need_grad=False)["E_total"])
        assert W[a, a] == pytest.approx(-(es[0] - es[1]) / (2 * h), rel=1e-6)


# ------------------------------------------------------------------ QEq
@pytest.mark.parametrize("name", ["petn464", "cluster300"])
def test_qeq_cg_equals_dense_cholesky_and_neutral(params, name):
    w = synth.workload(name)
    m = _model(params, w)
    L = m.lists(w["x"])
    Hd = m.qeq_matrix(w["x"], L).toarray()
    assert np.array_equal(Hd, Hd.T)
    assert np.linalg.eigvalsh(Hd).min() > 0.0
    a = m.qeq(w["x"], L, tol=1e-12)
    b = m.qeq_dense(w["x"], L)
    assert np.abs(a["q"] - b["q"]).max() < 1e-10
    assert abs(a["q"].sum()) < 1e-12 * len(w["x"])


def test_block_jacobi_pcg_special_cases_and_solution(params):
    """Block-Jacobi PCG (the solver variant): blocks of one atom are Jacobi (the iterates of
    pcg up to rounding), one block covering every atom is the exact inverse (one iteration), and the
    32-atom blocks reach the dense solution; the blocks tile each replica."""
    w = synth.workload("petn464")
    m = _model(params, w)
    L = m.lists(w["x"])
    Hm = m.qeq_matrix(w["x"], L)
    n = len(w["x"])
    chi = params["chi"][m.types]
    eta = params["eta"][m.types]
    b = -chi
    xj, itj = ro.pcg(Hm, b, eta, 1e-10, 500)
    x1, it1 = ro.pcg_block(Hm, b, ro.blocks_of([0, n], 1), 1e-10, 500)
    assert abs(it1 - itj) <= 1                          # 1/eta vs a 1x1 inverse: rounding only
    assert np.abs(x1 - xj).max() < 1e-9 * np.abs(xj).max()
    xa, ita = ro.pcg_block(Hm, b, [(0, n)], 1e-10, 500)
    assert ita == 1
    xd = np.linalg.solve(Hm.toarray(), b)
    assert np.abs(xa - xd).max() < 1e-9 * np.abs(xd).max()
    x32, it32 = ro.pcg_block(Hm, b, ro.blocks_of([0, n]), 1e-10, 500)
    assert np.abs(x32 - xd).max() < 1e-8 * np.abs(xd).max()
    assert it32 < itj
    assert ro.blocks_of([0, 70, 75]) == [(0, 32), (32, 64), (64, 70), (70, 75)]
    q_j = m.qeq(w["x"], L, tol=1e-10)["q"]
    q_b = m.qeq(w["x"], L, tol=1e-10, precond="block32")["q"]
    assert np.abs(q_j - q_b).max() < 1e-8


def test_gmres_solution_and_minimal_residual(params):
    """GMRES (comparison solver): reaches the dense solution with non-increasing residuals;
    unpreconditioned and unrestarted, its residual after k steps is the minimum over the
    Krylov space CG also searches, so never above CG's; a diagonal system converges in one
    Jacobi-preconditioned step."""
    w = synth.workload("petn464")
    m = _model(params, w)
    L = m.lists(w["x"])
    Hm = m.qeq_matrix(w["x"], L)
    chi = params["chi"][m.types]
    eta = params["eta"][m.types]
    b = -chi
    xg, itg, hist = ro.gmres(Hm, b, eta, 1e-10, 500, restart=500)
    xd = np.linalg.solve(Hm.toarray(), b)
    assert np.abs(xg - xd).max() < 1e-8 * np.abs(xd).max()
    assert np.all(np.diff(hist) <= 1e-12)                  # non-increasing residuals
    # CG residual history with the same (identity) preconditioner: GMRES is never above it
    res_cg = []
    x = np.zeros_like(b); r = b.copy(); p = r.copy(); rr = r @ r
    for _ in range(25):
        wv = Hm @ p; al = rr / (p @ wv); x = x + al * p; r = r - al * wv
        res_cg.append(np.linalg.norm(r) / np.linalg.norm(b))
        rr2 = r @ r; p = r + rr2 / rr * p; rr = rr2
    _, _, hist_id = ro.gmres(Hm, b, np.ones_like(eta), 1e-14, 25, restart=25)
    assert np.all(hist_id[1:26] <= np.array(res_cg) * (1 + 1e-9) + 1e-15)
    import scipy.sparse as sp
    D = sp.diags(eta)
    xd1, it1, _ = ro.gmres(D.tocsr(), b, eta, 1e-12, 10)
    assert it1 == 1 and np.abs(xd1 - b / eta).max() < 1e-12


def test_qeq_two_atom_closed_form(params):
    """Two atoms: q1 = -q2 = (chi2 - chi1) / (eta1 + eta2 - 2 H12)."""
    P = params
    box = np.array([40.0, 40.0, 40.0])
    x = np.array([[10.0, 10.0, 10.0], [13.1, 11.0, 9.5]])
    t = np.array([0, 3])
    m = oracle.Model(P, t, box, synth.OPTIONS_DEFAULT)
    L = m.lists(x)
    qq = m.qeq(x, L, tol=1e-14)["q"]
    r = np.linalg.norm(x[1] - x[0])
    g = P["gamma"][0, 3]
    xr = r / 10.0
    tap = 20 * xr ** 7 - 70 * xr ** 6 + 84 * xr ** 5 - 35 * xr ** 4 + 1
    h12 = tap * P["k_e"] / (r ** 3 + g ** -3) ** (1.0 / 3.0)
    q1 = (P["chi"][3] - P["chi"][0]) / (P["eta"][0] + P["eta"][3] - 2 * h12)
    assert qq[0] == pytest.approx(q1, rel=1e-12)
    assert qq[1] == pytest.approx(-q1, rel=1e-12)


def test_coulomb_plus_polarisation_is_the_qeq_quadratic_form(params, cluster_ref):
    """E_coul + E_pol (pair sum over the half list) = chi.q + 1/2 q^T H q (matrix form)."""
    w, ref = cluster_ref
    m = _model(params, w)
    Hd = m.qeq_matrix(w["x"], ref["lists"]).toarray()
    q = ref["qeq"]["q"]
    chi = params["chi"][w["types"]]
    quad = chi @ q + 0.5 * q @ Hd @ q
    assert ref["E"]["coul"] + ref["E"]["pol"] == pytest.approx(quad, rel=1e-11)


# ------------------------------------------------------------------ special geometries
def _chain4(theta, omega, b=1.40):
    """i-j-k-l with bond length b, both bond angles theta, dihedral omega (0 = cis)."""
    j = np.zeros(3)
    k = np.array([b, 0, 0])
    i = b * np.array([np.cos(theta), np.sin(theta), 0.0])
    l_ = k + b * np.array([-np.cos(theta), np.sin(theta) * np.cos(omega), np.sin(theta) * np.sin(omega)])
    return np.stack([i, j, k, l_]) + 15.0


@pytest.mark.parametrize("which,ratio", [
    ("V1", lambda w: (1 + np.cos(w)) / 2),
    ("V3", lambda w: (1 + np.cos(3 * w)) / 2),
])
def test_torsion_dihedral_dependence(params, which, ratio):
    """With a single cosine amplitude, fixed bonds and angles, E_tors(omega)/E_tors(0) is
    the textbook cosine ratio; omega = 0 is cis (pins the dihedral and its sign)."""
    P = _steep(params)
    for k in ("V1", "V2", "V3"):
        if k != which:
            P[k] = P[k] * 0.0
    P[which] = np.full((4, 4), 2.5)
    box = np.array([30.0, 30.0, 30.0])
    t = np.zeros(4, np.int64)
    m = oracle.Model(P, t, box, synth.OPTIONS_DEFAULT)
    th = np.deg2rad(110.0)
    e0 = None
    for w in np.deg2rad([0.0, 35.0, 60.0, 90.0, 150.0]):
        x = _chain4(th, w)
        L = m.lists(x)
        assert len(L["bond"]["i"]) == 3
        e = m.energy(x, np.zeros(4), L, need_grad=False, term_mask=("tors",))["E"]["tors"]
        if e0 is None:
            e0 = e
            assert e0 != 0.0
        else:
            assert e / e0 == pytest.approx(ratio(w), rel=1e-10, abs=1e-12)


def test_conjugation_dihedral_dependence(params):
    """E_conj at omega = 90 deg over omega = 0 is 1 - sin(th1) sin(th2)."""
    P = _steep(params)
    P["p_cot1"] = np.full((4, 4), -1.5)
    box = np.array([30.0, 30.0, 30.0])
    m = oracle.Model(P, np.zeros(4, np.int64), box, synth.OPTIONS_DEFAULT)
    th = np.deg2rad(115.0)
    es = []
    for w in (0.0, np.pi / 2):
        x = _chain4(th, w)
        es.append(m.energy(x, np.zeros(4), m.lists(x), need_grad=False, term_mask=("conj",))["E"]["conj"])
    assert es[1] / es[0] == pytest.approx(1 - np.sin(th) ** 2, rel=1e-10)


def test_hbond_angular_factor(params):
    """X-H...Z: E_hb(bent 90 deg)/E_hb(linear) = sin^4(45 deg)/sin^4(90 deg) = 1/4, at fixed
    H...Z distance; and the distance factor is 1 at r = r0hb."""
    P = _steep(params)
    box = np.array([30.0, 30.0, 30.0])
    t = np.array([3, 1, 3])                      # O - H ... O
    m = oracle.Model(P, t, box, synth.OPTIONS_DEFAULT)
    r0 = P["r0hb"][3, 3]
    es = []
    for ang in (np.pi, np.pi / 2):
        x = np.array([[0.0, 0, 0], [0.97, 0, 0], [0.97 + r0 * -np.cos(ang), r0 * np.sin(ang), 0]]) + 15.0
        L = m.lists(x)
        assert len(L["bond"]["i"]) == 1
        es.append(m.energy(x, np.zeros(3), L, need_grad=False, term_mask=("hbond",))["E"]["hbond"])
    assert es[1] / es[0] == pytest.approx(0.25, rel=1e-12)
    # linear, r = r0: E = p_hb1 (1 - exp(-p_hb2 BO)) exactly
    L = m.lists(np.array([[0.0, 0, 0], [0.97, 0, 0], [0.97 + r0, 0, 0]]) + 15.0)
    out = m.energy(np.array([[0.0, 0, 0], [0.97, 0, 0], [0.97 + r0, 0, 0]]) + 15.0, np.zeros(3), L,
                   need_grad=False, term_mask=("hbond",))
    bo = out["parts"]["bo"][0]
    assert es[0] == pytest.approx(P["p_hb1"][3, 3] * (1 - np.exp(-P["p_hb2"][3, 3] * bo)), rel=1e-12)


def test_vdw_well_depth(params):
    """Two atoms, van der Waals only: at the shielded distance f13 = rv the Morse-type
    bracket equals -1, so E_vdW = -D Tap(r)."""
    P = params
    a, b = 0, 3
    pv = P["p_vdW1"]
    rv, gw, D = P["vdw_rv"][a, b], P["vdw_gw"][a, b], P["vdw_D"][a, b]
    r = (rv ** pv - gw ** -pv) ** (1.0 / pv)
    box = np.array([40.0, 40.0, 40.0])
    x = np.array([[10.0, 10.0, 10.0], [10.0 + r, 10.0, 10.0]])
    m = oracle.Model(P, np.array([a, b]), box, synth.OPTIONS_DEFAULT)
    e = m.energy(x, np.zeros(2), m.lists(x), need_grad=False, term_mask=("vdw",))["E"]["vdw"]
    xr = r / 10.0
    tap = 20 * xr ** 7 - 70 * xr ** 6 + 84 * xr ** 5 - 35 * xr ** 4 + 1
    assert e == pytest.approx(-D * tap, rel=1e-12)


def test_valence_angle_energy_vanishes_at_its_minimum(params):
    """E_val = C (1 - exp(-p_val2 (theta0 - theta)^2)) >= 0 with minimum 0: scanning theta
    for a bent C-C-C molecule reaches 0 at an interior angle."""
    P = _steep(params)
    box = np.array([30.0, 30.0, 30.0])
    m = oracle.Model(P, np.zeros(3, np.int64), box, synth.OPTIONS_DEFAULT)
    es = []
    ths = np.deg2rad(np.linspace(80, 170, 361))
    for th in ths:
        x = np.array([[1.5 * np.cos(th), 1.5 * np.sin(th), 0], [0.0, 0, 0], [1.5, 0, 0]]) + 15.0
        es.append(m.energy(x, np.zeros(3), m.lists(x), need_grad=False, term_mask=("val",))["E"]["val"])
    es = np.array(es)
    assert es.min() >= 0.0
    assert es.min() < 1e-4 * es.max()
    assert 0 < np.argmin(es) < len(es) - 1


# ------------------------------------------------------------------ dynamics
def test_nve_energy_error_is_second_order_in_dt(params):
    """Velocity Verlet on a smooth energy (the tapered nonbonded terms with QEq charges)
    conserves energy up to O(dt^2): halving dt over the same time divides it by ~4."""
    w = synth.workload("cluster300")
    m = oracle.Model(params, w["types"], w["box"], dict(w["options"], qeq_tol=1e-12),
                     term_mask=("vdw", "coul", "pol"))
    e0 = m.forces(w["x"])["E_total"] + oracle.kinetic(w["v"], params["mass"][w["types"]])
    errs = []
    for dt, n in ((0.4, 2), (0.2, 4)):
        _, _, _, et = oracle.verlet(m, w["x"], w["v"], dt, n)
        errs.append(abs(et[-1] - e0))
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_nve_drift_full_energy_petn464(params):
    """Full energy (list thresholds included): 10 steps of 0.1 fs drift below 1e-4 relative."""
    w = synth.workload("petn464")
    m = _model(params, dict(w, options=dict(w["options"], qeq_tol=1e-10)))
    _, _, _, et = oracle.verlet(m, w["x"], w["v"], 0.1, 10)
    assert np.abs(et - et[0]).max() / abs(et[0]) < 1e-4


def test_verlet_free_particles_move_ballistically(params):
    """Atoms far apart (no interaction within the cutoffs, q = 0 forces vanish): one
    Verlet step is x + dt v exactly."""
    P = params_without(params, chi=1)
    box = np.array([80.0, 80.0, 80.0])
    x = np.array([[10.0, 10.0, 10.0], [50.0, 50.0, 50.0]])
    v = np.array([[0.01, -0.02, 0.03], [-0.01, 0.0, 0.005]])
    m = oracle.Model(P, np.array([0, 3]), box, synth.OPTIONS_DEFAULT)
    x1, v1, F, _ = oracle.verlet(m, x, v, 0.1, 1)
    assert np.abs(F).max() == 0.0
    assert np.array_equal(x1, x + 0.1 * v)
    assert np.array_equal(v1, v)


def test_free_flight_is_verlet_with_every_term_off():
    """Free flight equals the oracle's velocity Verlet on a model whose terms are all off
    (zero forces), bit for bit, and the straight line x + k dt v folded into the box."""
    P = synth.make_params()
    w = synth.workload("cluster150", temperature=3000.0)
    m = oracle.Model(P, w["types"], w["box"], w["options"], term_mask=())
    xv, vv, F, _ = oracle.verlet(m, w["x"], w["v"], 0.5, 6)
    assert np.all(F == 0.0) and np.array_equal(vv, w["v"])
    xf = oracle.free_flight(w["x"], w["v"], w["box"], 0.5, 6)
    assert np.array_equal(xf, xv)
    assert np.all((xf >= 0) & (xf < w["box"]))
    line = np.mod(w["x"] + 6 * 0.5 * w["v"], w["box"])
    d = xf - line
    d -= w["box"] * np.round(d / w["box"])
    assert np.abs(d).max() < 1e-12
    assert np.abs(xf - w["x"]).max() > 0.1                   # the atoms did move
