"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, on the same
seeded inputs.

Tolerances: lists bit-exact (sets of (i, j, image shift)); FP64 path max|dF|/RMS(F)
<= 1e-9 and energies to 1e-10 relative (rounding-order differences only); mixed path
max|dF|/RMS(F) <= 1e-5, |dE_tot|/|E_tot| <= 1e-6 and |dq| <= 1e-5 e.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

FP64_F, FP64_E = 1e-9, 1e-10
MIX_F, MIX_E, MIX_Q = 1e-5, 1e-6, 1e-5


@pytest.fixture(scope="module")
def rx():
    from paper_1706_07772_gb300 import build as B
    B.build()
    import paper_1706_07772_gb300.reaxff as m
    m.load()
    return m


@pytest.fixture(scope="module")
def params():
    return synth.make_params()


_REF = {}


def reference(params, name, tol=1e-12):
    key = (name, tol)
    if key not in _REF:
        w = synth.workload(name)
        o = dict(w["options"], qeq_tol=1e-10)
        m = oracle.Model(params, w["types"], w["box"], o)
        _REF[key] = (w, o, m, m.forces(w["x"], tol=tol))
    return _REF[key]


def make(rx, params, w, o, prec, **kw):
    c = rx.ReaxFF(params, w["types"], w["box"], o, precision=prec, **kw)
    c.set_state(w["x"], w["v"])
    return c


def keyset(i, j, s, n):
    return np.sort(oracle.sort_key(np.asarray(i, np.int64), np.asarray(j, np.int64), np.asarray(s, np.int64), n))


PRECS = [0, 1]
NAMES = ["petn464", "cluster300"]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", NAMES)
def test_lists_bit_exact(rx, params, name, prec):
    w, o, m, ref = reference(params, name)
    n = len(w["x"])
    c = make(rx, params, w, o, prec)
    c.build_lists()
    L = ref["lists"]
    B = L["bond"]
    want = {
        rx.LIST_FAR: keyset(L["far"]["i"], L["far"]["j"], L["far"]["s"], n),
        rx.LIST_BOND: keyset(np.concatenate([B["i"], B["j"]]), np.concatenate([B["j"], B["i"]]),
                             np.concatenate([B["s"], -B["s"]]), n),
        rx.LIST_HBOND: keyset(L["hbond"]["i"], L["hbond"]["j"], L["hbond"]["s"], n),
    }
    for which, k in want.items():
        got = keyset(*c.get_lists(which), n)
        assert len(got) == len(k) and np.array_equal(got, k), which
    c.close()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", NAMES)
def test_bond_orders(rx, params, name, prec):
    w, o, m, ref = reference(params, name)
    n = len(w["x"])
    c = make(rx, params, w, o, prec)
    c.forces(q=ref["qeq"]["q"])
    i, j, s = c.get_lists(rx.LIST_BOND)
    bo = c.get_bond_orders()
    B = ref["lists"]["bond"]
    okey = oracle.sort_key(B["i"], B["j"], B["s"], n)
    pos = {k: t for t, k in enumerate(okey)}
    canon = oracle.half_mask(i, j, s)
    gkey = oracle.sort_key(i[canon].astype(np.int64), j[canon].astype(np.int64), s[canon].astype(np.int64), n)
    idx = np.array([pos[k] for k in gkey])
    pr = ref["parts"]
    assert np.allclose(bo["bo_prime"][canon], pr["bo_prime"][idx], rtol=1e-12, atol=1e-15)
    tol = 1e-12 if prec == 0 else 2e-6
    for k_gpu, k_or in (("bo", "bo"), ("bo_pi", "bo_pi"), ("bo_pp", "bo_pp")):
        assert np.allclose(bo[k_gpu][canon], pr[k_or][idx], rtol=tol, atol=tol * 1e-3), k_gpu
    # bond orders are symmetric: both directions carry identical values
    full = oracle.sort_key(i.astype(np.int64), j.astype(np.int64), s.astype(np.int64), n)
    rev = oracle.sort_key(j.astype(np.int64), i.astype(np.int64), -s.astype(np.int64), n)
    where = {k: t for t, k in enumerate(full)}
    mirror = np.array([where[k] for k in rev])
    assert np.array_equal(bo["bo"], bo["bo"][mirror])
    c.close()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", NAMES)
def test_qeq_charges(rx, params, name, prec):
    w, o, m, ref = reference(params, name)
    c = make(rx, params, w, o, prec)
    q, its, itt, conv = c.qeq()
    assert conv
    dq = np.abs(q - ref["qeq"]["q"]).max()
    assert dq < (1e-8 if prec == 0 else MIX_Q)
    assert abs(q.sum()) < 1e-9 * len(q)
    c.close()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", NAMES)
def test_forces_energies_virial_fixed_charges(rx, params, name, prec):
    w, o, m, ref = reference(params, name)
    c = make(rx, params, w, o, prec)
    F, E, W = c.forces(q=ref["qeq"]["q"])
    rms = np.sqrt((ref["F"] ** 2).mean())
    ftol, etol = (FP64_F, FP64_E) if prec == 0 else (MIX_F, MIX_E)
    assert np.abs(F - ref["F"]).max() / rms < ftol
    assert abs(E[0].sum() - ref["E_total"]) < etol * abs(ref["E_total"])
    scale = sum(abs(v) for v in ref["E"].values())
    for k, t in enumerate(oracle.TERMS):
        assert abs(E[0][k] - ref["E"][t]) < max(etol * scale, 1e-9), t
    Wm = rx.virial_matrix(W[0])
    assert np.abs(Wm - ref["W"]).max() < (1e-9 if prec == 0 else 1e-5) * np.abs(ref["W"]).max()
    c.close()


@pytest.mark.parametrize("term", list(oracle.TERMS))
def test_per_term_forces_fp64(rx, params, term):
    """Each energy term's force alone (term mask) matches the gradient of that term."""
    w, o, m, ref = reference(params, "cluster300")
    qo = ref["qeq"]["q"]
    rt = m.energy(w["x"], qo, ref["lists"], term_mask=(term,))
    c = make(rx, params, w, o, 0, term_mask=rx.term_mask(term))
    F, E, W = c.forces(q=qo)
    scale = max(np.abs(rt["F"]).max(), 1.0)
    assert np.abs(F - rt["F"]).max() < 1e-10 * max(scale, 100.0)
    c.close()


@pytest.mark.parametrize("prec", PRECS)
def test_forces_with_gpu_qeq(rx, params, prec):
    """Full path including the GPU QEq at the workload's tolerance (1e-8 for petn464)."""
    w, o, m, ref = reference(params, "petn464")
    c = rx.ReaxFF(params, w["types"], w["box"], w["options"], precision=prec)
    c.set_state(w["x"], w["v"])
    F, E, W = c.forces()
    rms = np.sqrt((ref["F"] ** 2).mean())
    assert np.abs(F - ref["F"]).max() / rms < (1e-7 if prec == 0 else MIX_F)
    assert abs(E[0].sum() - ref["E_total"]) < (1e-9 if prec == 0 else MIX_E) * abs(ref["E_total"])
    _, _, q = c.get_state()
    assert np.abs(q - ref["qeq"]["q"]).max() < MIX_Q
    c.close()


def test_nve_trajectory_matches_oracle(rx, params):
    """10 velocity-Verlet steps (dt 0.1 fs) on petn464: FP64 GPU positions, velocities and
    per-step total energy against the oracle's own integrator."""
    w = synth.workload("petn464")
    o = dict(w["options"], qeq_tol=1e-10)
    m = oracle.Model(params, w["types"], w["box"], o)
    x, v, F, et = oracle.verlet(m, w["x"], w["v"], 0.1, 10)
    c = rx.ReaxFF(params, w["types"], w["box"], o, precision=0)
    c.set_state(w["x"], w["v"])
    eg = c.step(10, 0.1)
    xg, vg, _ = c.get_state()
    d = xg - x
    d -= w["box"] * np.round(d / w["box"])
    assert np.abs(d).max() < 1e-9
    assert np.abs(vg - v).max() < 1e-9
    assert np.abs(eg[:, 0] - et).max() < 1e-7 * abs(et[0])
    c.close()


def test_mixed_nve_drift_no_worse_than_fp64(rx, params):
    """40 NVE steps on petn464: the mixed path's drift max |E - E0| / |E0| is the FP64 path's
    up to rounding. The slack is 2 % of the FP64 drift plus 4e-7 for two energy evaluations
    at the mixed path's energy error (measured <= 2e-7 relative per evaluation). The energy
    curves also agree step by step to 1e-6."""
    w = synth.workload("petn464")
    drift, curves = [], []
    for prec in PRECS:
        c = rx.ReaxFF(params, w["types"], w["box"], w["options"], precision=prec)
        c.set_state(w["x"], w["v"])
        e = c.step(40, 0.1)[:, 0]
        curves.append(e)
        drift.append(np.abs(e - e[0]).max() / abs(e[0]))
        c.close()
    assert drift[0] < 1e-4
    assert drift[1] <= 1.02 * drift[0] + 4e-7, drift
    assert np.abs(curves[1] - curves[0]).max() < 1e-6 * abs(curves[0][0])


def test_bitwise_reproducible(rx, params):
    w = synth.workload("cluster300")
    outs = []
    for _ in range(2):
        c = rx.ReaxFF(params, w["types"], w["box"], w["options"], precision=1)
        c.set_state(w["x"], w["v"])
        outs.append(c.forces())
        c.close()
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)


def test_capacity_regrow(rx, params):
    """A far-list capacity below the densest row overflows and is regrown transparently."""
    w, o, m, ref = reference(params, "cluster300")
    c = make(rx, params, w, o, 0, capacity_margin=1.0)
    F, E, W = c.forces(q=ref["qeq"]["q"])
    rms = np.sqrt((ref["F"] ** 2).mean())
    assert np.abs(F - ref["F"]).max() / rms < FP64_F
    c.close()


def test_error_codes(rx, params):
    w = synth.workload("petn464")
    with pytest.raises(rx.ReaxFFError) as e:
        rx.ReaxFF(params, w["types"], np.array([9.0, 20.0, 20.0]), w["options"])
    assert e.value.code == rx.E_INVALID
    bad = dict(params, ntypes=0)
    with pytest.raises(rx.ReaxFFError):
        rx.ReaxFF(bad, w["types"], w["box"], w["options"])
    c = rx.ReaxFF(params, w["types"], w["box"], w["options"])
    with pytest.raises(rx.ReaxFFError) as e:
        c.forces()
    assert e.value.code == rx.E_STATE
    x = w["x"].copy()
    x[3, 1] = np.nan
    with pytest.raises(rx.ReaxFFError) as e:
        c.set_state(x)
    assert e.value.code == rx.E_NAN
    c.close()
    c = rx.ReaxFF(params, w["types"], w["box"], dict(w["options"], qeq_max_iter=1))
    c.set_state(w["x"])
    q, its, itt, conv = c.qeq()
    assert not conv and its[0] == 1
    c.close()


def test_batched_replicas_match_single_runs(rx, params):
    """Three uneven replicas in one context: per-replica energies and forces equal the
    single-system runs (no interaction crosses replicas)."""
    specs = [("petn464", 0), ("cluster300", 1), ("petn464", 2)]
    ws = [synth.workload(nm, seed=sd) for nm, sd in specs]
    types = np.concatenate([w["types"] for w in ws])
    x = np.concatenate([w["x"] for w in ws])
    off = np.cumsum([0] + [len(w["x"]) for w in ws])
    boxes = np.stack([w["box"] for w in ws])
    o = dict(ws[0]["options"], qeq_tol=1e-10)
    cb = rx.ReaxFF(params, types, boxes, o, precision=0, rep_offsets=off)
    cb.set_state(x)
    Fb, Eb, Wb = cb.forces()
    for r, w in enumerate(ws):
        c = rx.ReaxFF(params, w["types"], w["box"], o, precision=0)
        c.set_state(w["x"])
        F, E, W = c.forces()
        rms = np.sqrt((F ** 2).mean())
        assert np.abs(Fb[off[r]:off[r + 1]] - F).max() < 1e-8 * rms
        assert np.allclose(Eb[r], E[0], rtol=1e-9, atol=1e-8)
        c.close()
    cb.close()


@pytest.mark.parametrize("skin", [0.02, 1.0, -1.0])
def test_lists_stay_exact_along_md(rx, params, skin):
    """After steps that move atoms across box faces (3000 K velocities, every term off so
    that the positions are the host's own free flight, bit for bit) the far, bond and H-bond
    lists of the running context equal the oracle's lists at those positions, with the skin
    candidate list rebuilt often (0.02 A), rarely (1 A) or not used (< 0)."""
    w = synth.workload("cluster300", temperature=3000.0)
    n = len(w["x"])
    assert np.all((w["x"] >= 0) & (w["x"] < w["box"]))
    c = rx.ReaxFF(params, w["types"], w["box"], w["options"], precision=1, skin=skin, term_mask=rx.NO_TERMS)
    c.set_state(w["x"], w["v"])
    c.step(30, 0.5)
    xg, vg, _ = c.get_state()
    x = oracle.free_flight(w["x"], w["v"], w["box"], 0.5, 30)
    assert np.array_equal(xg, x) and np.array_equal(vg, w["v"])
    L = oracle.build_lists(x, w["types"], w["box"], params, w["options"])
    B = L["bond"]
    want = {
        rx.LIST_FAR: keyset(L["far"]["i"], L["far"]["j"], L["far"]["s"], n),
        rx.LIST_BOND: keyset(np.concatenate([B["i"], B["j"]]), np.concatenate([B["j"], B["i"]]),
                             np.concatenate([B["s"], -B["s"]]), n),
        rx.LIST_HBOND: keyset(L["hbond"]["i"], L["hbond"]["j"], L["hbond"]["s"], n),
    }
    for which, k in want.items():
        got = keyset(*c.get_lists(which), n)
        assert np.array_equal(got, k), which
    c.close()


def test_candidate_build_with_crowded_cells(rx, params):
    """A dense 4,200-atom cluster in a 21 A box has one candidate cell holding every atom. The
    candidate build then stages each stencil cell in several shared-memory passes (more than
    512 atoms) and gives each block more home atoms than one pass takes (more than 256 with
    16 blocks per cell). The far list it yields must be the one the cell stencil builds
    without candidates (skin < 0), as a set of (i, j, image) entries."""
    n, L = 4200, 21.0
    t, x, box = synth.random_cluster(n, (L, L, L), seed=7)
    o = dict(synth.OPTIONS_DEFAULT)
    got = []
    for skin in (0.7, -1.0):
        c = rx.ReaxFF(params, t, box, o, precision=1, skin=skin, term_mask=rx.NO_TERMS)
        c.set_state(x)
        c.build_lists()
        got.append(keyset(*c.get_lists(rx.LIST_FAR), n))
        c.close()
    assert len(got[0]) > 1500 * n
    assert np.array_equal(got[0], got[1])


def test_candidates_cover_pairs_two_cells_apart(rx, params):
    """Two atoms 10.6 A apart across two cell boundaries of a 10.5 A grid (box 31.5 A)
    fly towards each other by 0.35 A each (below the skin/2 rebuild trigger): the
    pair, now 9.9 A apart, must be in the far list. The candidate cells have to be at
    least r_nb + skin wide for the 27-cell stencil to have seen it at the build."""
    box = np.array([31.5, 31.5, 31.5])
    x = np.array([[10.45, 5.0, 5.0], [21.05, 5.0, 5.0]])
    v = np.array([[0.035, 0.0, 0.0], [-0.035, 0.0, 0.0]])
    types = np.array([0, 0], np.int32)
    o = dict(synth.OPTIONS_DEFAULT)
    c = rx.ReaxFF(params, types, box, o, precision=1, skin=1.0, term_mask=rx.NO_TERMS)
    c.set_state(x, v)
    c.step(20, 0.5)
    xg, _, _ = c.get_state()
    xf = oracle.free_flight(x, v, box, 0.5, 20)            # every term off: straight lines
    assert np.array_equal(xg, xf)
    assert abs(np.linalg.norm(xf[1] - xf[0]) - 9.9) < 0.01
    L = oracle.build_lists(xf, types, box, params, o)
    want = keyset(L["far"]["i"], L["far"]["j"], L["far"]["s"], 2)
    assert len(want) == 2                                  # (0, 1) and (1, 0), image shift 0
    got = keyset(*c.get_lists(rx.LIST_FAR), 2)
    assert np.array_equal(got, want)
    c.close()


def test_state_round_trip_keeps_the_trajectory(rx, params):
    """Downloading the state and uploading it unchanged between two calls of 5 steps gives
    the 10-step trajectory bit for bit (the unchanged positions keep forces, lists and the
    solution history); a moved atom is seen (forces equal a fresh context's at that state)."""
    w = synth.workload("petn464")
    a = rx.ReaxFF(params, w["types"], w["box"], w["options"], precision=1)
    a.set_state(w["x"], w["v"])
    ea = a.step(10, 0.1)
    xa, va, qa = a.get_state()
    b = rx.ReaxFF(params, w["types"], w["box"], w["options"], precision=1)
    b.set_state(w["x"], w["v"])
    eb1 = b.step(5, 0.1)
    x5, v5, _ = b.get_state()
    b.set_state(x5, v5)
    eb2 = b.step(5, 0.1)
    xb, vb, qb = b.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(qa, qb)
    assert np.array_equal(ea, np.concatenate([eb1, eb2]))
    xm = xb.copy()
    xm[0, 0] += 0.01
    b.set_state(xm, vb)
    q = synth.fixed_charges(len(xm), seed=3)
    Fb, Eb, _ = b.forces(q=q)
    c = rx.ReaxFF(params, w["types"], w["box"], w["options"], precision=1)
    c.set_state(xm, vb)
    Fc, Ec, _ = c.forces(q=q)
    assert np.array_equal(Fb, Fc) and np.array_equal(Eb, Ec)
    for ctx in (a, b, c):
        ctx.close()
