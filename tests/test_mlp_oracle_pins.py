"""Pins of the learned-warm-start oracle (descriptors, network, gradients, Adam) against
closed forms, invariances and finite differences -- no GPU."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as mo

BIG = np.array([40.0, 40.0, 40.0])


def _block(e):
    return slice(e * (mo.NR + mo.NA), (e + 1) * (mo.NR + mo.NA))


def test_radial_two_atoms_closed_form():
    r = 2.3
    x = np.array([[10.0, 10.0, 10.0], [10.0 + r, 10.0, 10.0]])
    types = np.array([0, 3])
    D = mo.descriptors(x, types, BIG)
    mu = mo.MU0 + np.arange(mo.NR) * (mo.MU1 - mo.MU0) / (mo.NR - 1)
    fc = 0.5 * (math.cos(math.pi * r / mo.RC_R) + 1.0)
    want = np.exp(-mo.ETA_R * (r - mu) ** 2) * fc
    assert np.allclose(D[0, _block(3)][:mo.NR], want, rtol=1e-13, atol=1e-15)
    assert np.allclose(D[1, _block(0)][:mo.NR], want, rtol=1e-13, atol=1e-15)
    # nothing else: other elements' blocks and (one neighbour) every angular feature
    mask = np.ones(mo.NF, bool)
    mask[_block(3)][:mo.NR] = False
    assert np.all(D[0][mask] == 0.0)


def test_angular_three_atoms_closed_form():
    a, b, th = 1.1, 1.4, math.radians(104.0)
    c0 = np.array([15.0, 15.0, 15.0])
    x = np.array([c0, c0 + [a, 0, 0], c0 + [b * math.cos(th), b * math.sin(th), 0]])
    types = np.array([3, 1, 0])           # centre O, neighbours H and C
    D = mo.descriptors(x, types, BIG)
    fa, fb = (0.5 * (math.cos(math.pi * r / mo.RC_A) + 1.0) for r in (a, b))
    for z, zeta in enumerate(mo.ZETAS):
        for k, eta in enumerate(mo.ETAS_A):
            for l, lam in enumerate(mo.LAMBDAS):
                v = 2.0 ** (1 - zeta) * (1 + lam * math.cos(th)) ** zeta * math.exp(-eta * (a * a + b * b)) * fa * fb
                f = mo.NR + 4 * z + 2 * k + l
                # the ordered pair (j=H, k=C) lands in the H block, (j=C, k=H) in the C block
                assert D[0, _block(1)][f] == pytest.approx(v, rel=1e-12)
                assert D[0, _block(0)][f] == pytest.approx(v, rel=1e-12)


def _cluster(seed, n=12):
    rng = np.random.default_rng(seed)
    x = 15.0 + rng.uniform(-2.0, 2.0, (n, 3))
    types = rng.integers(0, 4, n)
    return x, types


def test_descriptor_invariances():
    x, types = _cluster(3)
    D = mo.descriptors(x, types, BIG)
    # translation
    assert np.allclose(mo.descriptors(x + [0.7, -1.3, 2.1], types, BIG), D, rtol=1e-12, atol=1e-12)
    # rotation about the cluster centre
    q = np.linalg.qr(np.random.default_rng(5).normal(size=(3, 3)))[0]
    c = x.mean(0)
    assert np.allclose(mo.descriptors((x - c) @ q.T + c, types, BIG), D, rtol=1e-10, atol=1e-12)
    # permutation of the atoms permutes the rows
    p = np.random.default_rng(6).permutation(len(x))
    assert np.allclose(mo.descriptors(x[p], types[p], BIG), D[p], rtol=1e-12, atol=1e-12)
    # periodic wrap of one atom changes nothing
    xw = x.copy()
    xw[0, 0] += BIG[0]
    assert np.allclose(mo.descriptors(xw, types, BIG), D, rtol=1e-12, atol=1e-12)


def test_cutoffs_are_continuous():
    for rc, e in ((mo.RC_R, 0), (mo.RC_A, 1)):
        x = np.array([[10.0, 10.0, 10.0], [10.0 + rc - 1e-7, 10.0, 10.0], [10.0, 10.0 + 1.0, 10.0]])
        D = mo.descriptors(x, np.array([2, e, 1]), BIG)
        if rc == mo.RC_R:
            assert np.abs(D[0, _block(e)][:mo.NR]).max() < 1e-12
        else:
            assert np.abs(D[0, _block(e)][mo.NR:]).max() < 1e-12


def test_silu_gradient():
    z = np.linspace(-8, 8, 41)
    h = 1e-6
    fd = (mo.silu(z + h) - mo.silu(z - h)) / (2 * h)
    assert np.allclose(mo.silu_grad(z), fd, rtol=1e-8, atol=1e-10)


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(11)
    n = 9
    Xn = rng.normal(size=(n, mo.NF))
    types = np.array([0, 1, 2, 3, 0, 1, 2, 3, 0])
    q = rng.normal(scale=0.3, size=n)
    theta = rng.normal(scale=0.15, size=(mo.NT, mo.NPAR))
    L, g = mo.loss_and_grad(theta, Xn, types, q)
    for _ in range(40):
        t = rng.integers(0, mo.NT)
        k = rng.integers(0, mo.NPAR)
        h = 1e-6
        tp, tm = theta.copy(), theta.copy()
        tp[t, k] += h
        tm[t, k] -= h
        fd = (mo.loss_and_grad(tp, Xn, types, q)[0] - mo.loss_and_grad(tm, Xn, types, q)[0]) / (2 * h)
        assert g[t, k] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_forward_reduces_to_linear_model():
    """With W2 = identity-like through SiLU removed (W1 = W2 = 0), y = silu(b2) . w3 + b3."""
    theta = np.zeros((mo.NT, mo.NPAR))
    W1, b1, W2, b2, w3, b3 = mo.unpack(theta[2])
    b2 += 0.5
    w3 += 0.25
    theta[2, -1] = 0.125
    y, _ = mo.forward(theta, np.ones((3, mo.NF)), np.array([2, 2, 2]))
    assert np.allclose(y, mo.H2 * 0.25 * 0.5 / (1 + math.exp(-0.5)) + 0.125, rtol=1e-14)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(2)
    theta = rng.normal(size=50)
    g = rng.normal(size=50)
    lr, eps = 1e-3, 1e-8
    t1, m, v = mo.adam_step(theta, g, np.zeros(50), np.zeros(50), 1, lr, eps=eps)
    assert np.allclose(t1, theta - lr * g / (np.abs(g) + eps), rtol=1e-14, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_norm_stats():
    D = np.array([[1.0, 5.0, 0.0], [3.0, 5.0, 0.0]])
    mean, inv = mo.norm_stats(D)
    assert np.allclose(mean, [2.0, 5.0, 0.0]) and np.allclose(inv, [1.0, 0.0, 0.0])
