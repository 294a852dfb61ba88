"""Launch-schedule autotuner: picks among the stated alternatives, keeps results within
rounding of the default schedule, and reuses its cache file."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1])
def test_autotune_schedule_and_cache(params, tmp_path, prec):
    import paper_1706_07772_gb300.reaxff as rx
    w = synth.workload("petn464")
    c = rx.ReaxFF(params, w["types"], w["box"], w["options"], precision=prec)
    c.set_state(w["x"], w["v"])
    c.forces()
    _, _, q = c.get_state()
    F0, E0, _ = c.forces(q=q)                       # fixed charges: only the schedule changes
    x0, v0, _ = c.get_state()
    cache = tmp_path / "tune.txt"
    sch = c.autotune(cache)
    # the solve's placement is timed on MD steps, each candidate's steps rolled back: the
    # context's positions and velocities are the ones it had
    x1, v1, _ = c.get_state()
    assert np.array_equal(x1, x0) and np.array_equal(v1, v0)
    # torsion lanes 1 and angle lanes 4 are candidates of the second, overlapped tuning pass
    assert sch[0] in (1, 2, 4, 8) and sch[1] in (128, 256, 512) and sch[2] in (128, 256, 512)
    assert sch[3] in (128, 256, 512) and sch[4] in (64, 128, 256) and sch[5] in (64, 128, 256)
    assert sch[6] in (4, 8, 16, 32) and sch[7] in (0, 1, 2, 3, 4, 5)
    F1, E1, _ = c.forces(q=q)
    rms = np.sqrt((F0 ** 2).mean())
    assert np.abs(F1 - F0).max() < (1e-12 if prec == 0 else 1e-6) * rms
    assert np.allclose(E1, E0, rtol=1e-12 if prec == 0 else 1e-7)
    # a second context of the same system takes the schedule from the cache
    c2 = rx.ReaxFF(params, w["types"], w["box"], w["options"], precision=prec)
    c2.set_state(w["x"], w["v"])
    assert c2.autotune(cache) == sch
    assert len(cache.read_text().splitlines()) == 1
    c2.step(3, 0.1)
    c.step(3, 0.1)
    x1, _, _ = c.get_state()
    x2, _, _ = c2.get_state()
    assert np.abs(x1 - x2).max() < 1e-9
    c.close()
    c2.close()


def _system(name):
    """A named workload, or "batch3": three uneven crystal replicas in one context."""
    if name != "batch3":
        w = synth.workload(name)
        return w, {}
    parts = [synth.crystal(sh, seed=40 + r) for r, sh in enumerate(((2, 2, 2), (3, 2, 2), (2, 2, 3)))]
    types = np.concatenate([p[0] for p in parts])
    x = np.concatenate([p[1] for p in parts])
    v = np.concatenate([synth.velocities(p[0], 300.0, seed=50 + r) for r, p in enumerate(parts)])
    off = np.cumsum([0] + [len(p[0]) for p in parts])
    w = dict(types=types, x=x, v=v, box=np.stack([np.asarray(p[2], float) for p in parts]),
             options=dict(synth.OPTIONS_DEFAULT))
    return w, {"rep_offsets": off}


@pytest.mark.parametrize("name", ["petn464", "cluster300", "batch3"])
def test_qeq_beside_terms_matches_serial_order(params, tmp_path, name):
    """The QEq solve on the second stream beside the charge-free terms (schedule entry 7 = 1
    or 2: 512 or 256 threads on every SM; 3, 4, 5: 1024-thread blocks on 1/2, 3/8, 5/8 of the
    SMs, with their own chunks of rows) and before them (0) give the same MD trajectory,
    charges, forces and energies to within the solve tolerance (1e-6): the CG dot products'
    partial sums follow the thread count and the chunks, so a solve may stop one iteration
    apart."""
    import re

    import paper_1706_07772_gb300.reaxff as rx
    w, kw = _system(name)
    c = rx.ReaxFF(params, w["types"], w["box"], w["options"], precision=rx.MIXED, **kw)
    c.set_state(w["x"], w["v"])
    c.autotune(tmp_path / "tune.txt")
    c.close()
    line = (tmp_path / "tune.txt").read_text().strip()
    assert re.search(r"qov=[0-5]$", line)
    res = []
    for qov in (0, 1, 2, 3, 4, 5):
        f = tmp_path / ("tune%d.txt" % qov)
        f.write_text(re.sub(r"qov=[0-5]$", "qov=%d" % qov, line) + "\n")
        c = rx.ReaxFF(params, w["types"], w["box"], w["options"], precision=rx.MIXED, **kw)
        c.set_state(w["x"], w["v"])
        assert c.autotune(f)[7] == qov
        e = c.step(20, 0.1)
        x, v, q = c.get_state()
        F, E, _ = c.forces()
        res.append((e, x, v, q, F, E.sum(1)))
        c.close()
    e0, x0, v0, q0, F0, E0 = res[0]
    for e1, x1, v1, q1, F1, E1 in res[1:]:
        assert np.abs(x1 - x0).max() < 1e-8 and np.abs(v1 - v0).max() < 1e-8
        assert np.abs(q1 - q0).max() < 1e-5
        assert np.abs(F1 - F0).max() < 1e-5 * np.sqrt((F0 ** 2).mean())
        assert np.abs(e1 - e0).max() < 1e-7 * np.abs(e0).max()
        assert np.abs(E1 - E0).max() < 1e-7 * np.abs(E0).max()


def test_cache_line_out_of_range_is_retuned(params, tmp_path):
    """A cache line whose entries the tuner could not have picked (a solve shape past the last,
    a block size of 100) is ignored: the context is tuned again and the new line appended."""
    import re

    import paper_1706_07772_gb300.reaxff as rx
    w = synth.workload("petn464")
    c = rx.ReaxFF(params, w["types"], w["box"], w["options"], precision=rx.MIXED)
    c.set_state(w["x"], w["v"])
    good = tmp_path / "tune.txt"
    sch = c.autotune(good)
    line = good.read_text().strip()
    for bad_line in (re.sub(r"qov=[0-5]$", "qov=9", line), re.sub(r"nb=\d+", "nb=100", line)):
        f = tmp_path / "bad.txt"
        f.write_text(bad_line + "\n")
        s2 = c.autotune(f)
        assert s2[7] in (0, 1, 2, 3, 4, 5) and s2[1] in (128, 256, 512)
        lines = f.read_text().strip().splitlines()
        assert len(lines) == 2 and lines[0] == bad_line
    F, E, _ = c.forces()
    assert np.isfinite(F).all()
    assert len(sch) == 8
    c.close()
