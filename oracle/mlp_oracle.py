"""FP64 CPU oracle of the learned QEq warm start -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU legs may import this module. It
shares no code with the CUDA path.

The paper's QEq (Sec. 3.3) starts CG from an extrapolated guess; this project adds a
learned guess: a small per-atom network predicts each atom's charge from its local
environment, the CG then runs to the same tolerance (the guess only moves its starting
point). What this module computes, written from the definitions:

  * descriptors (192 per atom): for each neighbour element e (4),
      radial  G_R[e, k] = sum_{j of element e, r_ij < RC_R} exp(-ETA_R (r_ij - mu_k)^2) fc(r_ij)
              mu_k = MU0 + k (MU1 - MU0) / 31, k = 0..31, fc(r) = (cos(pi r / RC) + 1) / 2
      angular G_A[e, (z, a, l)] = 2^(1 - zeta_z) sum over ordered pairs of neighbour points
              (j, k), j != k, both within RC_A, j of element e:
              (1 + lambda_l cos theta_jik)^zeta_z exp(-eta_a (r_ij^2 + r_ik^2)) fc(r_ij) fc(r_ik)
              zeta in (1, 2, 4, 8), eta_a in (0.05, 0.3), lambda in (+1, -1)
    laid out per element as [32 radial, 16 angular] with angular index 4 z + 2 a + l;
    neighbours are all periodic images of all atoms within the cutoff
  * input normalisation x~ = (x - mean) * inv_std (statistics of the training set)
  * per centre element t an MLP 192 -> 64 -> 64 -> 1 with SiLU:
      z1 = x~ W1 + b1, a1 = silu(z1), z2 = a1 W2 + b2, a2 = silu(z2), y = a2 . w3 + b3
  * the mean-squared-error loss over atoms, its gradients by reverse-mode differentiation
    written out by hand, and one Adam step
"""
from __future__ import annotations

import math

import numpy as np

NT = 4                       # elements (C, H, N, O)
NR, NA = 32, 16              # radial and angular features per neighbour element
NF = NT * (NR + NA)          # 192
H1 = H2 = 64
RC_R, RC_A = 6.0, 3.5        # radial and angular cutoffs (A)
MU0, MU1 = 0.8, 6.0
ETA_R = 1.0 / (2.0 * ((MU1 - MU0) / (NR - 1)) ** 2)
ZETAS = (1.0, 2.0, 4.0, 8.0)
ETAS_A = (0.05, 0.3)
LAMBDAS = (1.0, -1.0)
# parameter layout of one element's network (float vector): W1[192][64], b1[64], W2[64][64],
# b2[64], w3[64], b3
NPAR = NF * H1 + H1 + H1 * H2 + H2 + H2 + 1   # 16,577


def fc(r, rc):
    """Cosine cutoff (cos(pi r / rc) + 1) / 2 inside rc, 0 outside."""
    return np.where(r < rc, 0.5 * (np.cos(np.pi * r / rc) + 1.0), 0.0)


def neighbour_points(x, box, i, rc):
    """All periodic images (j, shift) with 0 < |x_j + shift L - x_i| < rc; returns the
    atom indices and the vectors d = x_j + s L - x_i (brute force over 27 images)."""
    js, ds = [], []
    for sx in (-1, 0, 1):
        for sy in (-1, 0, 1):
            for sz in (-1, 0, 1):
                s = np.array([sx, sy, sz], float)
                d = (x - x[i]) + s * box
                r = np.sqrt((d * d).sum(1))
                m = (r < rc) & (r > 0.0)
                js.append(np.nonzero(m)[0])
                ds.append(d[m])
    return np.concatenate(js), np.concatenate(ds)


def descriptors(x, types, box):
    """192 descriptors per atom (definitions in the module docstring)."""
    x = np.asarray(x, float)
    n = len(x)
    mu = MU0 + np.arange(NR) * (MU1 - MU0) / (NR - 1)
    D = np.zeros((n, NF))
    for i in range(n):
        js, ds = neighbour_points(x, box, i, RC_R)
        r = np.sqrt((ds * ds).sum(1))
        g = np.exp(-ETA_R * (r[:, None] - mu[None, :]) ** 2) * fc(r, RC_R)[:, None]
        for e in range(NT):
            D[i, e * (NR + NA):e * (NR + NA) + NR] = g[types[js] == e].sum(0)
        m = r < RC_A
        ja, da, ra = js[m], ds[m], r[m]
        fa = fc(ra, RC_A)
        for p in range(len(ja)):                  # ordered pairs (p, q), p != q
            for q in range(len(ja)):
                if p == q:
                    continue
                c = float(da[p] @ da[q]) / (ra[p] * ra[q])
                e = types[ja[p]]
                base = e * (NR + NA) + NR
                for z, zeta in enumerate(ZETAS):
                    for a, eta in enumerate(ETAS_A):
                        rad = math.exp(-eta * (ra[p] ** 2 + ra[q] ** 2)) * fa[p] * fa[q]
                        for l, lam in enumerate(LAMBDAS):
                            D[i, base + 4 * z + 2 * a + l] += 2.0 ** (1.0 - zeta) * (1.0 + lam * c) ** zeta * rad
    return D


def norm_stats(D):
    """Per-feature mean and 1/std (0 where a feature is constant)."""
    mean = D.mean(0)
    std = D.std(0)
    inv = np.where(std > 1e-12, 1.0 / np.where(std > 1e-12, std, 1.0), 0.0)
    return mean, inv


def unpack(theta):
    """One element's parameter vector -> (W1, b1, W2, b2, w3, b3)."""
    o = 0
    W1 = theta[o:o + NF * H1].reshape(NF, H1); o += NF * H1
    b1 = theta[o:o + H1]; o += H1
    W2 = theta[o:o + H1 * H2].reshape(H1, H2); o += H1 * H2
    b2 = theta[o:o + H2]; o += H2
    w3 = theta[o:o + H2]; o += H2
    b3 = theta[o]
    return W1, b1, W2, b2, w3, b3


def _sigmoid(z):
    """Logistic function written without overflow: 1/(1 + e^-z) = (1 + tanh(z/2)) / 2."""
    return 0.5 * (1.0 + np.tanh(0.5 * z))


def silu(z):
    return z * _sigmoid(z)


def silu_grad(z):
    s = _sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def forward(theta, Xn, types):
    """theta: (NT, NPAR); Xn: normalised descriptors (n, 192). Returns y (n,) and the
    per-element caches for backward."""
    y = np.zeros(len(Xn))
    cache = {}
    for t in range(NT):
        idx = np.nonzero(types == t)[0]
        if len(idx) == 0:
            continue
        W1, b1, W2, b2, w3, b3 = unpack(theta[t])
        X = Xn[idx]
        z1 = X @ W1 + b1
        a1 = silu(z1)
        z2 = a1 @ W2 + b2
        a2 = silu(z2)
        y[idx] = a2 @ w3 + b3
        cache[t] = (idx, X, z1, a1, z2, a2)
    return y, cache


def loss_and_grad(theta, Xn, types, q):
    """L = mean over atoms of (y - q)^2 and dL/dtheta (NT, NPAR), reverse mode by hand."""
    y, cache = forward(theta, Xn, types)
    n = len(q)
    L = float(((y - q) ** 2).mean())
    g = np.zeros_like(theta)
    for t, (idx, X, z1, a1, z2, a2) in cache.items():
        W1, b1, W2, b2, w3, b3 = unpack(theta[t])
        dy = 2.0 * (y[idx] - q[idx]) / n
        dw3 = a2.T @ dy
        db3 = dy.sum()
        dz2 = np.outer(dy, w3) * silu_grad(z2)
        dW2 = a1.T @ dz2
        db2 = dz2.sum(0)
        dz1 = (dz2 @ W2.T) * silu_grad(z1)
        dW1 = X.T @ dz1
        db1 = dz1.sum(0)
        g[t] = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dw3, [db3]])
    return L, g


def adam_step(theta, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
