"""Learned QEq warm start on the GPU against the oracle (oracle/mlp_oracle.py):
descriptors, the BF16 tensor-core forward, FP32 loss/gradients, Adam, and training."""
import numpy as np
import pytest

import oracle
import synth
from oracle import mlp_oracle as mo

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rx():
    import paper_1706_07772_gb300.reaxff as rx
    rx.load()
    return rx


def _ctx(rx, params, name):
    w = synth.workload(name)
    c = rx.ReaxFF(params, w["types"], w["box"], w["options"], precision=rx.MIXED)
    c.set_state(w["x"], w["v"])
    return w, c


@pytest.mark.parametrize("name", ["petn464", "cluster300"])
def test_descriptors_match_oracle(rx, params, name):
    w, c = _ctx(rx, params, name)
    D = c.mlp_descriptors()
    Dref = mo.descriptors(w["x"], np.asarray(w["types"]), np.asarray(w["box"], float))
    assert D.shape == Dref.shape
    err = np.abs(D - Dref)
    assert np.all(err <= 1e-4 * np.abs(Dref) + 2e-5), float((err / (np.abs(Dref) + 1e-3)).max())
    c.close()


def _bf16(a):
    """Round float32 to bfloat16 (round to nearest even) and back."""
    a = np.ascontiguousarray(a, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def _rand_theta(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    th = np.zeros((mo.NT, mo.NPAR))
    for t in range(mo.NT):
        W1, b1, W2, b2, w3, b3 = mo.unpack(th[t])
        W1[:] = rng.normal(size=W1.shape) * np.sqrt(1.0 / mo.NF) * scale
        b1[:] = rng.normal(size=b1.shape) * 0.1
        W2[:] = rng.normal(size=W2.shape) * np.sqrt(1.0 / mo.H1) * scale
        b2[:] = rng.normal(size=b2.shape) * 0.1
        w3[:] = rng.normal(size=w3.shape) * np.sqrt(1.0 / mo.H2)
        th[t, -1] = rng.normal() * 0.1
    return th


def _emulate_tc(theta, Xn, types):
    """The tensor-core forward's arithmetic: BF16 x~, W1, a1, W2; FP32 accumulation."""
    y = np.zeros(len(Xn))
    for t in range(mo.NT):
        idx = np.nonzero(types == t)[0]
        if len(idx) == 0:
            continue
        W1, b1, W2, b2, w3, b3 = (np.asarray(a, np.float64) for a in mo.unpack(theta[t].astype(np.float32).astype(np.float64)))
        X = _bf16(Xn[idx]).astype(np.float64)
        z1 = X @ _bf16(W1).astype(np.float64) + b1
        a1 = _bf16(mo.silu(z1)).astype(np.float64)
        z2 = a1 @ _bf16(W2).astype(np.float64) + b2
        y[idx] = mo.silu(z2) @ w3 + b3
    return y


def test_tensor_core_forward(rx, params):
    w, c = _ctx(rx, params, "petn464")
    types = np.asarray(w["types"])
    D = mo.descriptors(w["x"], types, np.asarray(w["box"], float))
    mean, inv = mo.norm_stats(D)
    theta = _rand_theta(7)
    c.mlp_set_params(theta, mean, inv)
    # the context keeps float32 statistics: normalise exactly as it does
    m32, i32 = mean.astype(np.float32), inv.astype(np.float32)
    Xn = ((D.astype(np.float32) - m32) * i32).astype(np.float32)
    y = c.mlp_infer(D.astype(np.float32), types)
    ref_bf16 = _emulate_tc(theta, Xn, types)
    ref64, _ = mo.forward(theta, (D - mean) * inv, types)
    scale = np.abs(ref64).max()
    # same rounding as the tensor cores: only the accumulation order differs
    assert np.abs(y - ref_bf16).max() < 1e-3 * scale, np.abs(y - ref_bf16).max() / scale
    # against the FP64 definition: BF16 operand error
    assert np.abs(y - ref64).max() < 2e-2 * scale
    # more atoms than one tile per element and a ragged tail, random order of elements
    rng = np.random.default_rng(3)
    m = 1000
    Dm = rng.normal(size=(m, mo.NF)).astype(np.float32) * 2.0 + 1.0
    tm = rng.integers(0, 4, m).astype(np.int32)
    ym = c.mlp_infer(Dm, tm)
    Xm = ((Dm - m32) * i32).astype(np.float32)
    ref = _emulate_tc(theta, Xm, tm)
    assert np.abs(ym - ref).max() < 1e-3 * np.abs(ref).max()
    c.close()


def test_loss_and_gradients_match_oracle(rx, params):
    w, c = _ctx(rx, params, "petn464")
    types = np.asarray(w["types"])
    D = mo.descriptors(w["x"], types, np.asarray(w["box"], float))
    mean, inv = mo.norm_stats(D)
    theta = _rand_theta(9)
    c.mlp_set_params(theta, mean, inv)
    q = np.random.default_rng(4).normal(scale=0.3, size=len(types))
    L, g = c.mlp_loss_grad(D.astype(np.float32), types, q.astype(np.float32))
    Xn = (D.astype(np.float32) - mean.astype(np.float32)) * inv.astype(np.float32)
    Lref, gref = mo.loss_and_grad(theta.astype(np.float32).astype(np.float64), Xn.astype(np.float64), types,
                                  q.astype(np.float32).astype(np.float64))
    assert L == pytest.approx(Lref, rel=1e-5)
    for t in range(mo.NT):
        assert np.abs(g[t] - gref[t]).max() <= 1e-4 * np.abs(gref[t]).max() + 1e-9, t
    c.close()


def test_adam_matches_oracle(rx, params):
    w, c = _ctx(rx, params, "petn464")
    theta = _rand_theta(12).astype(np.float32)
    c.mlp_set_params(theta, np.zeros(mo.NF, np.float32), np.ones(mo.NF, np.float32))
    rng = np.random.default_rng(5)
    th, m, v = theta.astype(np.float64), np.zeros_like(theta, np.float64), np.zeros_like(theta, np.float64)
    for step in (1, 2, 3):
        g = rng.normal(size=theta.shape).astype(np.float32) * 1e-3
        c.mlp_adam_step(g, 1e-3)
        th, m, v = mo.adam_step(th, g.astype(np.float64), m, v, step, 1e-3)
    got, _, _ = c.mlp_get_params()
    assert np.abs(got - th).max() < 1e-6
    c.close()


def test_training_learns_charges(rx, params):
    """Snapshots of an MD run of the method itself; the trained network predicts the
    charges of a later state far better than the per-element mean."""
    w, c = _ctx(rx, params, "petn464")
    c.mlp_reserve(12)
    c.mlp_init(1234)
    for _ in range(12):
        c.step(2, 0.1)
        c.mlp_collect()
    loss0 = None
    for ep in (1, 60):
        loss = c.mlp_train(ep, 2e-3)
        loss0 = loss if loss0 is None else loss0
    c.step(5, 0.1)
    _, _, q = c.get_state()
    qp = c.mlp_predict()
    types = np.asarray(w["types"])
    base = np.array([q[types == t].mean() for t in range(4)])[types]
    assert loss < 0.5 * loss0
    assert np.sqrt(((qp - q) ** 2).mean()) < 0.5 * np.sqrt(((base - q) ** 2).mean())
    c.close()


def test_learned_guess_saves_iterations_and_keeps_charges(rx, params):
    """Cold start (no solution history) on a held-out state: the learned guess for s cuts
    the CG iterations against the zero start, and the charges stay those of the solve."""
    w = synth.workload("petn464")
    c = rx.ReaxFF(params, w["types"], w["box"], w["options"], precision=rx.MIXED, warm_start=rx.WARM_MLP)
    c.set_state(w["x"], w["v"])
    c.mlp_reserve(16)
    c.mlp_init(99)
    for _ in range(16):
        c.step(2, 0.1)
        c.mlp_collect()
    c.mlp_train(80, 2e-3)
    theta, mean, inv = c.mlp_get_params()
    c.close()
    w2 = synth.workload("petn464", seed=7)                 # other jitter and velocities
    cs = rx.ReaxFF(params, w2["types"], w2["box"], w2["options"], precision=rx.MIXED, warm_start=rx.WARM_ZERO)
    cs.set_state(w2["x"], w2["v"])
    cs.step(10, 0.1)
    x2, v2, _ = cs.get_state()
    cs.close()
    # the zero-start reference is a fresh context at that state, so that its lists (and the
    # order of each row's entries, hence the FP32 SpMV rounding) are built as the learned
    # context's are
    cz = rx.ReaxFF(params, w2["types"], w2["box"], w2["options"], precision=rx.MIXED, warm_start=rx.WARM_ZERO)
    cz.set_state(x2, v2)
    qz, itz, ttz, _ = cz.qeq()
    cm = rx.ReaxFF(params, w2["types"], w2["box"], w2["options"], precision=rx.MIXED, warm_start=rx.WARM_MLP)
    cm.mlp_set_params(theta, mean, inv)
    cm.set_state(x2, v2)
    qm, itm, ttm, _ = cm.qeq()
    assert cm.qeq_warm_choice()[0] == 1
    assert itm[0] < itz[0], (itm, itz)
    assert ttm[0] == ttz[0]                                 # t starts at zero in both
    assert np.abs(qm - qz).max() < 1e-5
    assert abs(qm.sum()) < 1e-9 * len(qm)
    cz.close()
    cm.close()


def test_learned_guess_only_without_history(rx, params):
    """The learned start runs only for a solve without a usable solution history: the cold
    solve keeps it, while the steps that follow use the extrapolated start. Their solves then
    run the same SpMVs as a context with the extrapolated start, so no probe SpMV of the learned
    guess is added per step (that would be 10 extra over 10 steps). After a history reset the
    next solve takes the learned guess again."""
    w = synth.workload("petn464")
    c = rx.ReaxFF(params, w["types"], w["box"], w["options"], precision=rx.MIXED, warm_start=rx.WARM_MLP)
    c.set_state(w["x"], w["v"])
    c.mlp_reserve(16)
    c.mlp_init(99)
    for _ in range(16):
        c.step(2, 0.1)
        c.mlp_collect()
    c.mlp_train(80, 2e-3)
    theta, mean, inv = c.mlp_get_params()
    c.close()
    w2 = synth.workload("petn464", seed=7)
    cm = rx.ReaxFF(params, w2["types"], w2["box"], w2["options"], precision=rx.MIXED, warm_start=rx.WARM_MLP)
    cm.mlp_set_params(theta, mean, inv)
    ce = rx.ReaxFF(params, w2["types"], w2["box"], w2["options"], precision=rx.MIXED, warm_start=rx.WARM_EXTRAP)
    for cc in (cm, ce):
        cc.set_state(w2["x"], w2["v"])
        cc.qeq()
    assert cm.qeq_warm_choice()[0] == 1
    sp = []
    for cc in (cm, ce):
        s0 = cc.qeq_spmv_total()
        cc.step(10, 0.1)
        sp.append(cc.qeq_spmv_total() - s0)
    assert cm.qeq_warm_choice()[0] == 0
    assert sp[0] <= sp[1] + 2, sp
    cm.reset_qeq_history()
    cm.qeq()
    assert cm.qeq_warm_choice()[0] == 1
    cm.close()
    ce.close()
