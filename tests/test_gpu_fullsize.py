"""GPU parity at the full sizes of the benchmark workloads, in the launch configuration the
benchmark times: extrapolated warm start, Jacobi QEq at the workload tolerance (1e-6),
1 A Verlet-skin candidate lists, autotuned launch schedules.

petn32k (32,480 atoms), the whole system against the oracle:
  * far, bond and H-bond lists as sorted sets of (i, j, image shift), bit-exact;
  * QEq charges, |dq| <= 1e-5 e, and neutrality;
  * forces, per-term energies and the virial at the oracle's charges;
  * the lists again after 40 steps of free flight (every term masked off: the positions are
    the host's own x + dt v sequence, hot velocities), which takes the candidate list
    through reuse and rebuilds on the device.

petn1m (1,039,360 atoms), 1,000 sampled atoms in four regions, each evaluated by the oracle on
a cut-out deep enough that every quantity the sampled atoms depend on is exact
(oracle/cutout.py):
  * the far, bond and H-bond rows of the sampled atoms, bit-exact;
  * their forces at seeded fixed charges;
  * the QEq optimality condition chi_i + (H q)_i = mu on their rows at the charges the GPU
    solved for (a property of the solution: the oracle's matrix rows are applied to the GPU's
    answer; no expected value comes from the GPU), within the bound the CG stopping rule
    ||b - Hx|| <= tol ||b|| per system gives, plus the FP32 rounding of H on the mixed path.

Tolerances as in the small-system parity tests: FP64 max|dF|/RMS(F) <= 1e-9, mixed <= 1e-5,
|dE_tot|/|E_tot| <= 1e-6 (mixed), |dq| <= 1e-5 e.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import cutout

pytestmark = pytest.mark.gpu

PRECS = [0, 1]
MIX_F, MIX_E, MIX_Q = 1e-5, 1e-6, 1e-5
FP64_F, FP64_E = 1e-9, 1e-10


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


def keyset(i, j, s, n):
    return np.sort(oracle.sort_key(np.asarray(i, np.int64), np.asarray(j, np.int64), np.asarray(s, np.int64), n))


def bench_ctx(rx, params, w, prec, **kw):
    """A context as the benchmark makes it (extrapolated warm start, Jacobi QEq, default
    0.7 A skin, autotuned schedules)."""
    c = rx.ReaxFF(params, w["types"], w["box"], w["options"], precision=prec, warm_start=rx.WARM_EXTRAP,
                  qeq_precond=rx.PRECOND_JACOBI, **kw)
    c.set_state(w["x"], w["v"])
    c.autotune(None)
    return c


def oracle_keysets(L, n):
    B = L["bond"]
    return dict(far=keyset(L["far"]["i"], L["far"]["j"], L["far"]["s"], n),
                bond=keyset(np.concatenate([B["i"], B["j"]]), np.concatenate([B["j"], B["i"]]),
                            np.concatenate([B["s"], -B["s"]]), n),
                hbond=keyset(L["hbond"]["i"], L["hbond"]["j"], L["hbond"]["s"], n))


def gpu_keysets(rx, c, n, rows=None):
    """The context's lists as key sets; with `rows` (a boolean mask over atoms) only the rows
    of those atoms."""
    out = {}
    for name, which in (("far", rx.LIST_FAR), ("bond", rx.LIST_BOND), ("hbond", rx.LIST_HBOND)):
        i, j, s = c.get_lists(which)
        if rows is not None:
            sel = rows[i]
            i, j, s = i[sel], j[sel], s[sel]
        out[name] = keyset(i, j, s, n)
        del i, j, s
    return out


# ------------------------------------------------------------------------------ petn32k
@pytest.fixture(scope="module")
def ref32k(params):
    w = synth.workload("petn32k")
    o = dict(w["options"], qeq_tol=1e-10)
    m = oracle.Model(params, w["types"], w["box"], o)
    return w, m, m.forces(w["x"], tol=1e-10)


@pytest.mark.parametrize("prec", PRECS)
def test_petn32k_lists_bit_exact(rx, params, ref32k, prec):
    w, m, ref = ref32k
    n = len(w["x"])
    c = bench_ctx(rx, params, w, prec)
    c.build_lists()
    got = gpu_keysets(rx, c, n)
    want = oracle_keysets(ref["lists"], n)
    for k in want:
        assert len(got[k]) == len(want[k]) and np.array_equal(got[k], want[k]), k
    c.close()


@pytest.mark.parametrize("prec", PRECS)
def test_petn32k_qeq_charges(rx, params, ref32k, prec):
    w, m, ref = ref32k
    c = bench_ctx(rx, params, w, prec)
    q, its, itt, conv = c.qeq()
    assert conv
    assert np.abs(q - ref["qeq"]["q"]).max() < MIX_Q
    assert abs(q.sum()) < 1e-9 * len(q)
    c.close()


@pytest.mark.parametrize("prec", PRECS)
def test_petn32k_forces_energies_virial(rx, params, ref32k, prec):
    w, m, ref = ref32k
    c = bench_ctx(rx, params, w, prec)
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


def test_petn32k_lists_after_free_flight(rx, params):
    """40 steps of 0.5 fs at 3000 K velocities with every term off: the device positions
    equal the host's free flight bit for bit, and the lists the running context holds equal
    the oracle's lists at those positions (candidates reused between rebuilds)."""
    w = synth.workload("petn32k", temperature=3000.0)
    n = len(w["x"])
    assert np.all((w["x"] >= 0) & (w["x"] < w["box"]))
    c = bench_ctx(rx, params, w, 1, term_mask=rx.NO_TERMS)
    c.step(40, 0.5)
    xg, vg, _ = c.get_state()
    xh = oracle.free_flight(w["x"], w["v"], w["box"], 0.5, 40)
    assert np.array_equal(vg, w["v"])
    assert np.array_equal(xg, xh)
    d = (xh - w["x"] + 0.5 * w["box"]) % w["box"] - 0.5 * w["box"]
    moved = np.sqrt((d * d).sum(1)).max()
    assert moved > 0.5                                    # beyond skin/2: the candidates were rebuilt
    L = oracle.build_lists(xh, w["types"], w["box"], params, w["options"])
    got = gpu_keysets(rx, c, n)
    want = oracle_keysets(L, n)
    for k in want:
        assert np.array_equal(got[k], want[k]), k
    c.close()


# ------------------------------------------------------------------------------ petn1m
NREG, PER_REG = 4, 250


@pytest.fixture(scope="module")
def ref1m(params):
    """Seeded fixed charges, four sampled regions and the oracle's values on each."""
    w = synth.workload("petn1m")
    n = len(w["x"])
    o = w["options"]
    q = synth.fixed_charges(n, seed=7)
    D = cutout.dependency_radius(params, o)
    rng = np.random.default_rng(1706)
    regs = []
    for _ in range(NREG):
        centre = rng.uniform(0.0, 1.0, 3) * w["box"]
        ids, rr = cutout.region(w["x"], w["box"], centre, PER_REG)
        cu = cutout.Cutout(params, w["types"], w["x"], w["box"], o, centre, rr + D)
        rows = cutout.list_rows(w["x"], w["types"], w["box"], params, o, ids, cu.ids)
        regs.append(dict(ids=ids, cu=cu, F=cu.forces(q, ids), rows=rows))
    sample = np.zeros(n, bool)
    for r in regs:
        sample[r["ids"]] = True
    assert sample.sum() == NREG * PER_REG                  # regions do not overlap
    Fs = np.concatenate([r["F"] for r in regs])
    return dict(w=w, q=q, regs=regs, sample=sample, rms=np.sqrt((Fs ** 2).mean()))


@pytest.mark.parametrize("prec", PRECS)
def test_petn1m_sampled_rows_forces_and_qeq(rx, params, ref1m, prec):
    w, regs = ref1m["w"], ref1m["regs"]
    n = len(w["x"])
    c = bench_ctx(rx, params, w, prec)
    c.build_lists()
    got = gpu_keysets(rx, c, n, rows=ref1m["sample"])
    for name in ("far", "bond", "hbond"):
        want = np.sort(np.concatenate([keyset(r["rows"][name]["i"], r["rows"][name]["j"], r["rows"][name]["s"], n)
                                       for r in regs]))
        assert len(got[name]) == len(want) and np.array_equal(got[name], want), name
    # forces at the seeded fixed charges
    F, E, W = c.forces(q=ref1m["q"])
    ftol = FP64_F if prec == 0 else MIX_F
    for r in regs:
        assert np.abs(F[r["ids"]] - r["F"]).max() / ref1m["rms"] < ftol
    # QEq optimality on the sampled rows at the GPU's charges
    q, its, itt, conv = c.qeq()
    assert conv
    assert abs(q.sum()) < 1e-9 * n
    chi = np.asarray(params["chi"])[w["types"]]
    rho, mag = [], []
    for r in regs:
        a, b = r["cu"].qeq_rows(q, r["ids"])
        rho.append(a)
        mag.append(b)
    rho, mag = np.concatenate(rho), np.concatenate(mag)
    mu = rho.mean()          # within [mu - B, mu + B] with the true mu; minimises the RMS below
    tol = w["options"]["qeq_tol"]
    # |rho_i - mu| <= ||r_s|| + |mu| ||r_t|| + |(dH q)_i|, with ||r_s|| <= tol ||chi||,
    # ||r_t|| <= tol sqrt(n); dH = the rounding of H on the path (FP32 values: a few ulp)
    eps_h = 1e-15 if prec == 0 else 16.0 * 2.0 ** -24
    bound = tol * (np.linalg.norm(chi) + abs(mu) * np.sqrt(n)) + eps_h * mag
    assert np.all(np.abs(rho - mu) <= 2.0 * bound)
    # the residual's RMS over the sampled rows against its RMS bound over all rows
    rms_bound = tol * (np.sqrt((chi ** 2).mean()) + abs(mu)) + eps_h * mag.max()
    assert np.sqrt(((rho - mu) ** 2).mean()) <= 4.0 * rms_bound
    c.close()


def test_petn32k_1000_step_nve_mixed_no_worse_than_fp64(rx, params):
    """1000 NVE steps of 0.1 fs on petn32k (QEq tol 1e-6, extrapolated start) on both paths:
    the mixed path's total-energy drift is no worse than the FP64 path's, and the two energy
    curves agree step by step (measured: max |E - E0| / |E0| 4.487e-4 on both)."""
    w = synth.workload("petn32k")
    e = {}
    for prec in PRECS:
        c = rx.ReaxFF(params, w["types"], w["box"], w["options"], precision=prec, warm_start=rx.WARM_EXTRAP)
        c.set_state(w["x"], w["v"])
        e[prec] = c.step(1000, 0.1)[:, 0]
        c.close()
    drift = {p: np.abs(e[p] - e[p][0]).max() / abs(e[p][0]) for p in PRECS}
    assert drift[1] <= 1.02 * drift[0] + 1e-7, drift
    assert np.abs(e[1] - e[0]).max() < 1e-5 * abs(e[0][0])
