"""QEq initial-guess predictors (host function of the library, no GPU): predictor 0 is
Lagrange extrapolation (cubic for s, quadratic for t); predictors 1 and 2 are least-squares
cubics over the last 6 or 8 solutions: they reproduce the Lagrange weights up to four stored
solutions, equal an independent least-squares fit beyond, are exact on cubics and reproduce
constants."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def rx():
    import paper_1706_07772_gb300.reaxff as rx
    try:
        rx.load()
    except (ImportError, OSError) as e:
        pytest.skip("library not built: %s" % e)
    return rx


LAGR = {1: [1.0], 2: [2.0, -1.0], 3: [3.0, -3.0, 1.0], 4: [4.0, -6.0, 4.0, -1.0]}


@pytest.mark.parametrize("pred,window", [(1, 6), (2, 8)])
def test_least_squares_predictors(rx, pred, window):
    w = rx.extrap_weights(pred)
    assert w.shape == (2, 9, 8)
    assert np.all(w[:, 0] == 0.0)
    for sys in (0, 1):
        for m in range(1, 9):
            npt = min(m, window)
            row = w[sys, m]
            assert np.all(row[npt:] == 0.0)
            assert abs(row.sum() - 1.0) < 1e-12
            if npt <= 4:
                assert np.allclose(row[:npt], LAGR[npt], atol=1e-12)
            t = -np.arange(1, npt + 1, dtype=float)
            V = np.vander(t, min(npt - 1, 3) + 1, increasing=True)
            assert np.allclose(row[:npt], np.linalg.pinv(V)[0], atol=1e-12)
            if npt >= 4:
                c = np.random.default_rng(m).normal(size=4)
                xk = np.polyval(c[::-1], t)                 # a cubic sampled at t = -1..-npt
                assert abs(row[:npt] @ xk - c[0]) < 1e-11 * (1 + np.abs(c).sum())


def test_lagrange_predictor(rx):
    w = rx.extrap_weights(0)
    for m in range(1, 9):
        ks = LAGR[min(m, 4)]
        kt = LAGR[min(m, 3)]
        assert np.allclose(w[0, m, :len(ks)], ks) and np.all(w[0, m, len(ks):] == 0.0)
        assert np.allclose(w[1, m, :len(kt)], kt) and np.all(w[1, m, len(kt):] == 0.0)
    with pytest.raises(rx.ReaxFFError):
        rx.extrap_weights(3)
