"""Oracle values for sampled atoms of a large periodic system -- TEST INFRASTRUCTURE ONLY.

Only tests/ may use this module. Like the rest of the oracle it shares no code with the CUDA
path; it evaluates the plain oracle (reaxff_oracle.Model) on a spherical cut-out around the
sampled atoms, so that forces, list rows and QEq rows of a million-atom system can be
checked one region at a time.

Why a cut-out gives exact forces (the ReaxFF terms of Sec. 2.1, as the oracle writes them).
Let b be the longest possible bond: the largest r < r_bond with BO'(r) >= bo_cut over all
type pairs (every BO' component decays monotonically with r for p_bo1, p_bo3, p_bo5 < 0 and
p_bo2, p_bo4, p_bo6 > 0, which bond_reach() checks). Then, with B(k, rho) the ball of radius
rho around atom k:
  * BO'_kl depends on r_kl; Delta'_k on B(k, b); the corrected BO_kl on Delta'_k, Delta'_l,
    i.e. on B(k, 2b); Delta_k, Delta_lp,k and the other atom sums of corrected BO on B(k, 2b);
  * S_k (over/under-coordination) sums Delta_j - Delta_lp,j over bonded j: B(k, 3b), so
    E_over,k and E_under,k depend on B(k, 3b);
  * a valence angle (centre j) uses the BO of j's bonds, Delta_ang,j and, in the coalition
    term, the BO sums of the two end atoms: B(j, 3b); a torsion on central bond j-k uses BO
    of i-j, j-k, k-l and Delta_ang of j and k: B(j, 3b);
  * an H-bond X-H...Z uses BO_XH (B(H, 2b)) and Z within r_hb of H;
  * vdW, Coulomb (fixed charges) and the QEq matrix are pairwise within r_nb.
A term whose support contains atom i is therefore evaluated exactly when every atom within
max(6b, r_hb + 2b, r_nb) of i is present: dependency_radius(). Atoms further out change
no force on i; near the cut-out's surface forces are wrong, and only the inner atoms are
compared.

List rows are decided by their definition on the GLOBAL coordinates (d = (x_j - x_i) + s L
and r^2 rounded as the list definition fixes it), so membership is bit-exact whatever the
cut-out frame; the cut-out only bounds the candidates.
"""
from __future__ import annotations

import numpy as np

from oracle.reaxff_oracle import SHIFTS, Model, _r2, bo_prime_np


def bond_reach(P, opts, grid=200001):
    """Longest distance at which any type pair can still be bonded (BO' >= bo_cut), from a
    fine grid on [0, r_bond] (each component of BO' is decreasing in r, checked here, so the
    set of bonded distances is an interval starting at 0)."""
    r_bond, bo_cut = opts["r_bond"], opts["bo_cut"]
    for a, e in (("p_bo1", "p_bo2"), ("p_bo3", "p_bo4"), ("p_bo5", "p_bo6")):
        if not (np.all(np.asarray(P[a]) < 0) and np.all(np.asarray(P[e]) > 0)):
            raise ValueError("BO' is not decreasing in r for every type pair")
    r = np.linspace(0.0, r_bond, grid)[1:]
    nt = np.asarray(P["r0s"]).shape[0]
    reach = 0.0
    for ta in range(nt):
        for tb in range(nt):
            bs, bp, bpp = bo_prime_np(r, np.full(r.shape, ta), np.full(r.shape, tb), P, bo_cut)
            ok = np.nonzero(bs + bp + bpp >= bo_cut)[0]
            if len(ok):
                # the next grid point is not bonded: the reach is below it
                reach = max(reach, r[min(ok.max() + 1, len(r) - 1)])
    return reach


def dependency_radius(P, opts):
    """Radius around an atom that holds every atom its force depends on (module docstring)."""
    b = bond_reach(P, opts)
    return max(6.0 * b, opts["r_hb"] + 2.0 * b, opts["r_nb"])


def _min_image(d, box):
    return d - box * np.round(d / box)


def region(x, box, centre, m):
    """The m atoms nearest to the point `centre` (minimum image) and the largest of their
    distances."""
    d = _min_image(np.asarray(x, float) - centre, box)
    r = np.sqrt((d * d).sum(1))
    ids = np.argsort(r, kind="stable")[:m]
    return np.sort(ids), float(r[ids].max())


class Cutout:
    """Atoms within `radius` of `centre` (minimum image), unwrapped into one open cluster
    and placed in a box large enough that no periodic image of the cluster comes within
    r_nb of it; `model` is the oracle on that cluster."""

    def __init__(self, P, types, x, box, opts, centre, radius):
        x = np.asarray(x, float)
        box = np.asarray(box, float)
        if 2.0 * radius >= box.min():
            raise ValueError("cut-out diameter must be below every box length (unique images)")
        d = _min_image(x - centre, box)
        self.ids = np.nonzero((d * d).sum(1) < radius * radius)[0]
        side = 2.0 * radius + opts["r_nb"] + 1.0
        self.box = np.full(3, side)
        self.x = d[self.ids] + side / 2.0
        self.types = np.asarray(types)[self.ids]
        self.local = {int(g): k for k, g in enumerate(self.ids)}
        self.model = Model(P, self.types, self.box, opts)

    def index(self, gids):
        return np.array([self.local[int(g)] for g in gids], np.int64)

    def forces(self, q_global, gids):
        """Oracle forces on the atoms gids (global ids) at fixed global charges q_global."""
        out = self.model.forces(self.x, q=np.asarray(q_global, float)[self.ids])
        return out["F"][self.index(gids)]

    def qeq_rows(self, q_global, gids):
        """(chi + H q)_i and sum_j |H_ij q_j| (diagonal included) for the atoms gids."""
        if not hasattr(self, "_H"):
            self._H = self.model.qeq_matrix(self.x, self.model.lists(self.x))
        H = self._H
        q = np.asarray(q_global, float)[self.ids]
        k = self.index(gids)
        rows = H[k]
        chi = self.model.P["chi"][self.types[k]]
        return chi + rows @ q, abs(rows) @ np.abs(q)


def list_rows(x, types, box, P, opts, rows, candidates):
    """Far, bond and H-bond rows of the atoms `rows` (global ids), by the list definitions:
    far: all (j, s), s in {-1,0,1}^3, (j, s) != (i, 0), with r^2 < r_nb^2;
    bond: r^2 < r_bond^2 and BO'sig + BO'pi + BO'pp >= bo_cut;
    H-bond: i with hb flag 1, j with hb flag 2, r^2 < r_hb^2.
    `candidates` must hold every atom within r_nb of each row atom. Returns three dicts
    (i, j, s) in global ids, each row's entries in (j, s) order."""
    x = np.asarray(x, float)
    box = np.asarray(box, float)
    types = np.asarray(types)
    cand = np.asarray(candidates, np.int64)
    rn2, rb2, rh2 = opts["r_nb"] ** 2, opts["r_bond"] ** 2, opts["r_hb"] ** 2
    hb = np.asarray(P["hb"])
    out = {k: ([], [], []) for k in ("far", "bond", "hbond")}
    for i in np.asarray(rows, np.int64):
        # candidates near i by minimum image (a superset: 0.5 A margin), then every image
        d = _min_image(x[cand] - x[i], box)
        near = cand[(d * d).sum(1) < (opts["r_nb"] + 0.5) ** 2]
        jj = np.repeat(near, len(SHIFTS))
        ss = np.tile(SHIFTS, (len(near), 1))
        ii = np.full(len(jj), i)
        r2 = _r2(x, box, ii, jj, ss)
        keep = (r2 < rn2) & ~((jj == i) & ~ss.any(1))
        jj, ss, r2 = jj[keep], ss[keep], r2[keep]
        o = np.lexsort((ss[:, 2], ss[:, 1], ss[:, 0], jj))
        jj, ss, r2 = jj[o], ss[o], r2[o]
        ii = np.full(len(jj), i)
        out["far"][0].append(ii)
        out["far"][1].append(jj)
        out["far"][2].append(ss)
        bc = r2 < rb2
        bs, bp, bpp = bo_prime_np(np.sqrt(r2[bc]), types[ii[bc]], types[jj[bc]], P, opts["bo_cut"])
        kb = bs + bp + bpp >= opts["bo_cut"]
        out["bond"][0].append(ii[bc][kb])
        out["bond"][1].append(jj[bc][kb])
        out["bond"][2].append(ss[bc][kb])
        hm = (hb[types[i]] == 1) & (hb[types[jj]] == 2) & (r2 < rh2)
        out["hbond"][0].append(ii[hm])
        out["hbond"][1].append(jj[hm])
        out["hbond"][2].append(ss[hm])
    res = {}
    for k, (a, b, c) in out.items():
        res[k] = dict(i=np.concatenate(a) if a else np.zeros(0, np.int64),
                      j=np.concatenate(b) if b else np.zeros(0, np.int64),
                      s=np.concatenate(c) if c else np.zeros((0, 3), np.int64))
    return res
