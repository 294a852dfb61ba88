"""Plain FP64 CPU oracle of one ReaxFF timestep -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs
may import this module. It shares no code with the CUDA path.

What it computes (ReaxFF workflow of Sec. 2.1 and Fig. 1; list construction, pairwise
terms, 3-body/4-body enumeration and QEq of Sec. 3.3):
  * far-neighbour list (brute force and cell-binned), bond list, H-bond list
  * uncorrected and corrected bond orders, atom over/under-coordination quantities
  * the 13 energy terms: bond, lp, over, under, val, pen, coa, tors, conj, hbond,
    vdW, coul, pol
  * QEq: two Jacobi-preconditioned CG solves on the tapered H matrix, q = s - mu t; a
    block-Jacobi preconditioned variant (blocks of 32 consecutive atoms) with the same result;
    restarted GMRES as a comparison solver
  * forces F = -dE/dx at fixed charges and the virial -dE/d(strain), both by reverse-mode
    differentiation of the energy as written (plain definition of a force)
  * velocity Verlet

The paper names these terms but gives no formulas (Sec. 2.1); the functional forms are
the standard published ReaxFF forms as read for this project (each function says which
term it is). Everything is float64; plain loops / vectorised numpy / torch CPU ops.
"""
from __future__ import annotations

import math

import numpy as np
import torch

TERMS = ("bond", "lp", "over", "under", "val", "pen", "coa", "tors", "conj", "hbond",
         "vdw", "coul", "pol")
ACC_CONV = 4.184e-4      # (kcal/mol/A)/amu -> A/fs^2
_DT = torch.float64


# --------------------------------------------------------------------------------------
# taper (Sec. 3.3 "truncated electrostatics"; 7th-order taper of the ReaxFF literature)
# --------------------------------------------------------------------------------------
TAPER_COEF = (1.0, 0.0, 0.0, 0.0, -35.0, 84.0, -70.0, 20.0)   # in powers of x = r / R


def taper(r, R):
    """Tap(r) = 20x^7 - 70x^6 + 84x^5 - 35x^4 + 1, x = r/R (Horner form)."""
    x = r / R
    t = TAPER_COEF[7]
    for c in TAPER_COEF[6::-1]:
        t = t * x + c
    return t


# --------------------------------------------------------------------------------------
# neighbour lists (Sec. 3.3 "Neighbor and Interaction Lists")
# --------------------------------------------------------------------------------------
SHIFTS = np.array([[sx, sy, sz] for sx in (-1, 0, 1) for sy in (-1, 0, 1) for sz in (-1, 0, 1)],
                  np.int64)


def _r2(x, box, i, j, s):
    """r^2 exactly as the list definition fixes it: d = (xj - xi) + s*L per component,
    r^2 = (dx*dx + dy*dy) + dz*dz, separate IEEE roundings (no fused multiply-add)."""
    d = (x[j] - x[i]) + s * box
    return (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]


def far_list_bruteforce(x, box, rc):
    """All ordered (i, j, s) with r^2 < rc^2 over every atom pair and the 27 image shifts,
    excluding the atom itself at s = 0. Needs every box length > rc (|s_k| <= 1 then
    covers every image in range)."""
    x = np.asarray(x, float)
    box = np.asarray(box, float)
    n = len(x)
    out_i, out_j, out_s = [], [], []
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ii, jj = ii.ravel(), jj.ravel()
    for s in SHIFTS:
        ss = np.broadcast_to(s, (len(ii), 3))
        r2 = _r2(x, box, ii, jj, ss)
        keep = r2 < rc * rc
        if not s.any():
            keep &= ii != jj
        out_i.append(ii[keep])
        out_j.append(jj[keep])
        out_s.append(ss[keep])
    return np.concatenate(out_i), np.concatenate(out_j), np.concatenate(out_s)


def far_list_cells(x, box, rc):
    """Same set as far_list_bruteforce, found through a cell grid with cells >= rc and a
    27-cell stencil with periodic image shifts (the cell-binned far list)."""
    x = np.asarray(x, float)
    box = np.asarray(box, float)
    nc = np.maximum(np.floor(box / rc).astype(np.int64), 1)
    c = np.minimum(np.floor(x / box * nc).astype(np.int64), nc - 1)
    cid = (c[:, 2] * nc[1] + c[:, 1]) * nc[0] + c[:, 0]
    order = np.argsort(cid, kind="stable")
    ncell = int(nc.prod())
    start = np.searchsorted(cid[order], np.arange(ncell + 1))
    out_i, out_j, out_s = [], [], []
    for cz in range(nc[2]):
        for cy in range(nc[1]):
            for cx in range(nc[0]):
                a = order[start[(cz * nc[1] + cy) * nc[0] + cx]:start[(cz * nc[1] + cy) * nc[0] + cx + 1]]
                if len(a) == 0:
                    continue
                for o in SHIFTS:
                    t = np.array([cx, cy, cz]) + o
                    s = np.floor_divide(t, nc)               # image shift of the wrapped cell
                    t = t - s * nc
                    b = order[start[(t[2] * nc[1] + t[1]) * nc[0] + t[0]]:start[(t[2] * nc[1] + t[1]) * nc[0] + t[0] + 1]]
                    if len(b) == 0:
                        continue
                    ii = np.repeat(a, len(b))
                    jj = np.tile(b, len(a))
                    ss = np.broadcast_to(s, (len(ii), 3))
                    r2 = _r2(x, box, ii, jj, ss)
                    keep = r2 < rc * rc
                    if not s.any():
                        keep &= ii != jj
                    out_i.append(ii[keep])
                    out_j.append(jj[keep])
                    out_s.append(np.array(ss[keep]))
    # with fewer than 3 cells along an axis, several stencil offsets reach the same
    # (cell, shift); keep each (i, j, s) once
    i = np.concatenate(out_i)
    j = np.concatenate(out_j)
    s = np.concatenate(out_s)
    key = ((i * len(x) + j) * 27 + ((s[:, 0] + 1) * 9 + (s[:, 1] + 1) * 3 + (s[:, 2] + 1)))
    _, u = np.unique(key, return_index=True)
    return i[u], j[u], s[u]


def sort_key(i, j, s, n):
    """Canonical integer key of (i, j, s) for set comparison of lists."""
    s = np.asarray(s)
    return (np.asarray(i, np.int64) * n + np.asarray(j, np.int64)) * 27 + \
        ((s[:, 0] + 1) * 9 + (s[:, 1] + 1) * 3 + (s[:, 2] + 1))


def half_mask(i, j, s):
    """Canonical half of a full list: i < j, or i == j with s lexicographically > 0."""
    s = np.asarray(s)
    lex = (s[:, 0] > 0) | ((s[:, 0] == 0) & ((s[:, 1] > 0) | ((s[:, 1] == 0) & (s[:, 2] > 0))))
    return (i < j) | ((i == j) & lex)


# --------------------------------------------------------------------------------------
# uncorrected bond order BO' and the bond list (Sec. 3.3; Table 2 "Init. Forces")
# --------------------------------------------------------------------------------------
def bo_prime_np(r, ti, tj, P, bo_cut):
    """Uncorrected sigma/pi/pi-pi bond orders (numpy, float64) before the bo_cut shift:
    BO'sig = (1 + bo_cut) exp(p_bo1 (r/r0s)^p_bo2); BO'pi = exp(p_bo3 (r/r0p)^p_bo4);
    BO'pp = exp(p_bo5 (r/r0pp)^p_bo6); a component is 0 where its r0 <= 0."""
    r0s, r0p, r0pp = P["r0s"][ti, tj], P["r0p"][ti, tj], P["r0pp"][ti, tj]
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        bs = np.where(r0s > 0, (1.0 + bo_cut) * np.exp(P["p_bo1"][ti, tj] * np.power(r / np.where(r0s > 0, r0s, 1), P["p_bo2"][ti, tj])), 0.0)
        bp = np.where(r0p > 0, np.exp(P["p_bo3"][ti, tj] * np.power(r / np.where(r0p > 0, r0p, 1), P["p_bo4"][ti, tj])), 0.0)
        bpp = np.where(r0pp > 0, np.exp(P["p_bo5"][ti, tj] * np.power(r / np.where(r0pp > 0, r0pp, 1), P["p_bo6"][ti, tj])), 0.0)
    return bs, bp, bpp


def build_lists(x, types, box, P, opts, brute=None):
    """Far list (full), bond list (unordered, canonical half) and H-bond list.

    bond membership: r^2 < r_bond^2 and BO'sig + BO'pi + BO'pp >= bo_cut (float64).
    H-bond list: for H atoms (hb flag 1), partners Z with hb flag 2 and r^2 < r_hb^2.
    """
    x = np.asarray(x, float)
    box = np.asarray(box, float)
    n = len(x)
    if brute is None:
        brute = n <= 600
    fi, fj, fs = (far_list_bruteforce if brute else far_list_cells)(x, box, opts["r_nb"])
    o = np.argsort(sort_key(fi, fj, fs, n), kind="stable")
    fi, fj, fs = fi[o], fj[o], fs[o]
    r2 = _r2(x, box, fi, fj, fs)
    # bond candidates from the canonical half
    h = half_mask(fi, fj, fs) & (r2 < opts["r_bond"] ** 2)
    bi, bj, bsft = fi[h], fj[h], fs[h]
    r = np.sqrt(r2[h])
    bs, bp, bpp = bo_prime_np(r, types[bi], types[bj], P, opts["bo_cut"])
    tot = bs + bp + bpp
    keep = tot >= opts["bo_cut"]
    bond = dict(i=bi[keep], j=bj[keep], s=bsft[keep], bo_raw=tot[keep])
    # H-bond partner list
    hb = P["hb"]
    m = (hb[types[fi]] == 1) & (hb[types[fj]] == 2) & (r2 < opts["r_hb"] ** 2)
    hbl = dict(i=fi[m], j=fj[m], s=fs[m])
    return dict(far=dict(i=fi, j=fj, s=fs), bond=bond, hbond=hbl, n=n)


# --------------------------------------------------------------------------------------
# interaction enumeration (Sec. 3.3 "Three-body Interactions"; 4-body from bonds)
# --------------------------------------------------------------------------------------
def _directed(bond, n):
    """Directed bond entries grouped by centre: (centre, other, bond id, sign, shift of
    other relative to centre)."""
    nb = len(bond["i"])
    c = np.concatenate([bond["i"], bond["j"]])
    o = np.concatenate([bond["j"], bond["i"]])
    b = np.concatenate([np.arange(nb), np.arange(nb)])
    sg = np.concatenate([np.ones(nb), -np.ones(nb)])
    sh = np.concatenate([bond["s"], -bond["s"]])
    order = np.lexsort((o, c))
    c, o, b, sg, sh = c[order], o[order], b[order], sg[order], sh[order]
    start = np.searchsorted(c, np.arange(n + 1))
    return dict(c=c, o=o, b=b, sg=sg, sh=sh, start=start)


def enumerate_angles(D, n):
    """All (centre j; entry a, entry b) with a < b among the bond entries of j."""
    cnt = np.diff(D["start"])
    ea, eb = [], []
    for m in np.unique(cnt):
        if m < 2:
            continue
        centres = np.nonzero(cnt == m)[0]
        ta, tb = np.triu_indices(m, 1)
        base = D["start"][centres][:, None]
        ea.append((base + ta[None, :]).ravel())
        eb.append((base + tb[None, :]).ravel())
    if not ea:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    return np.concatenate(ea), np.concatenate(eb)


def enumerate_torsions(D, bond, n):
    """All (central bond b = (j, k) oriented j = its i-end, k = its j-end; entry a of j
    other than b; entry c of k other than b). Returns entry indices (a, c) and bond ids."""
    nb = len(bond["i"])
    side = (D["sg"] < 0).astype(np.int64)
    ent = np.empty(2 * nb, np.int64)
    ent[D["b"] * 2 + side] = np.arange(2 * nb)       # global entry index of (bond, side)
    j, k = bond["i"], bond["j"]
    cnt_all = np.diff(D["start"])
    cj, ck = cnt_all[j] - 1, cnt_all[k] - 1
    cnt = cj * ck
    tot = int(cnt.sum())
    if tot == 0:
        z = np.zeros(0, np.int64)
        return z, z, z
    bid = np.repeat(np.arange(nb), cnt)
    t = np.arange(tot) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    ia, ic = t // ck[bid], t % ck[bid]
    pj = ent[bid * 2] - D["start"][j[bid]]           # slot of b inside j's entries
    pk = ent[bid * 2 + 1] - D["start"][k[bid]]       # slot of b inside k's entries
    ea = D["start"][j[bid]] + ia + (ia >= pj)
    ec = D["start"][k[bid]] + ic + (ic >= pk)
    return ea, ec, bid


# --------------------------------------------------------------------------------------
# energy (all 13 terms) as a differentiable function of x (and strain)
# --------------------------------------------------------------------------------------
def _t(a):
    return torch.as_tensor(np.asarray(a), dtype=_DT)


def _sig(u):
    """1 / (1 + exp(u))."""
    return torch.sigmoid(-u)


class Model:
    """One system: parameters, types, box, options, with lists built for positions x."""

    def __init__(self, P, types, box, opts, term_mask=None):
        self.term_mask = term_mask
        self.P = P
        self.types = np.asarray(types, np.int64)
        self.box = np.asarray(box, float)
        self.opts = dict(opts)
        self.n = len(self.types)
        if np.any(self.box <= self.opts["r_nb"]):
            raise ValueError("every box length must exceed the nonbonded cutoff")

    # ---------------------------------------------------------------- lists
    def lists(self, x, brute=None):
        return build_lists(x, self.types, self.box, self.P, self.opts, brute=brute)

    # ---------------------------------------------------------------- QEq matrix
    def qeq_entries(self, x, fi, fj, fs):
        """Off-diagonal QEq matrix entry of each far-list entry (i, j, s):
        Tap(r) k_e / (r^3 + gamma_ij^-3)^(1/3), r = |x_j + s L - x_i| (Sec. 3.3 "QEq")."""
        P = self.P
        x = np.asarray(x, float)
        d = (x[fj] - x[fi]) + np.asarray(fs) * self.box
        r = np.sqrt((d * d).sum(1))
        g = P["gamma"][self.types[fi], self.types[fj]]
        return taper(r, self.opts["r_nb"]) * P["k_e"] / np.cbrt(r ** 3 + g ** -3.0)

    def qeq_matrix(self, x, L):
        """Sparse H (scipy CSR): H_ii = eta_i; H_ij = sum over images in range of
        Tap(r) k_e / (r^3 + gamma_ij^-3)^(1/3) (Sec. 3.3 "QEq")."""
        import scipy.sparse as sp
        P = self.P
        fi, fj, fs = L["far"]["i"], L["far"]["j"], L["far"]["s"]
        v = self.qeq_entries(x, fi, fj, fs)
        n = self.n
        Hm = sp.csr_matrix((v, (fi, fj)), shape=(n, n))
        Hm = Hm + sp.diags(P["eta"][self.types])
        return Hm.tocsr()

    def qeq(self, x, L, tol=None, max_iter=1000, guess=None, precond="jacobi"):
        """QEq charges via two PCG solves: H s = -chi, H t = -1; q = s - (sum s / sum t) t.
        precond "jacobi": M = diag(H), the paper's choice (Sec. 3.3); "block32": block
        Jacobi over 32 consecutive atoms (pcg_block), a solver variant with the same result.

        Convergence per system: ||b - H x||_2 / ||b||_2 <= tol (residual updated recursively
        inside CG). Returns dict(q, s, t, iters_s, iters_t)."""
        tol = self.opts["qeq_tol"] if tol is None else tol
        Hm = self.qeq_matrix(x, L)
        chi = self.P["chi"][self.types]
        eta = self.P["eta"][self.types]
        s0, t0 = (None, None) if guess is None else guess
        if precond == "block32":
            blocks = blocks_of([0, self.n])
            s, its = pcg_block(Hm, -chi, blocks, tol, max_iter, s0)
            t, itt = pcg_block(Hm, -np.ones(self.n), blocks, tol, max_iter, t0)
        else:
            s, its = pcg(Hm, -chi, eta, tol, max_iter, s0)
            t, itt = pcg(Hm, -np.ones(self.n), eta, tol, max_iter, t0)
        mu = s.sum() / t.sum()
        return dict(q=s - mu * t, s=s, t=t, iters_s=its, iters_t=itt, mu=mu)

    def qeq_dense(self, x, L):
        """Same charges from a dense Cholesky solve of both systems (small n only)."""
        Hd = self.qeq_matrix(x, L).toarray()
        chi = self.P["chi"][self.types]
        Lc = np.linalg.cholesky(Hd)
        sol = np.linalg.solve(Lc.T, np.linalg.solve(Lc, np.stack([-chi, -np.ones(self.n)], 1)))
        s, t = sol[:, 0], sol[:, 1]
        return dict(q=s - s.sum() / t.sum() * t, s=s, t=t)

    # ---------------------------------------------------------------- energy
    def energy(self, x, q, L, need_grad=True, term_mask=None):
        """Energy terms at positions x (n,3) and fixed charges q.

        Returns dict(E={term: float}, F=(n,3) forces, W=(3,3) virial -dE/d(strain),
        parts={...} intermediate float64 arrays for inspection)."""
        P, o, ty = self.P, self.opts, self.types
        n = self.n
        box = _t(self.box)
        X = torch.tensor(np.asarray(x, float), dtype=_DT, requires_grad=need_grad)
        EPS = torch.zeros(3, 3, dtype=_DT, requires_grad=need_grad)
        strain = torch.eye(3, dtype=_DT) + EPS

        def dvec(i, j, s):
            # interaction vector (xj - xi + s L), then homogeneous strain (I + eps)
            return ((X[j] - X[i]) + _t(s) * box) @ strain.T

        E = {}
        parts = {}
        mask = set(TERMS if term_mask is None else term_mask)

        # ---------------- bond orders (uncorrected, then corrected)
        B = L["bond"]
        bi, bj = B["i"], B["j"]
        nb = len(bi)
        db = dvec(bi, bj, B["s"])
        rb = torch.sqrt((db * db).sum(1))
        ti, tj = ty[bi], ty[bj]
        bo_cut = o["bo_cut"]

        def comp(r0, pa, pb, scale):
            r0 = _t(r0)
            ok = r0 > 0
            r0s = torch.where(ok, r0, torch.ones_like(r0))
            v = scale * torch.exp(_t(pa) * torch.pow(rb / r0s, _t(pb)))
            return torch.where(ok, v, torch.zeros_like(v))

        bs = comp(P["r0s"][ti, tj], P["p_bo1"][ti, tj], P["p_bo2"][ti, tj], 1.0 + bo_cut)
        bp = comp(P["r0p"][ti, tj], P["p_bo3"][ti, tj], P["p_bo4"][ti, tj], 1.0)
        bpp = comp(P["r0pp"][ti, tj], P["p_bo5"][ti, tj], P["p_bo6"][ti, tj], 1.0)
        bop = bs + bp + bpp - bo_cut                 # shifted total BO'
        bos_p = bs - bo_cut                          # shifted sigma part (unused further)
        del bos_p
        ones_b = torch.ones(nb, dtype=_DT)

        def atom_sum(v):
            out = torch.zeros(n, dtype=_DT)
            out = out.index_add(0, torch.as_tensor(bi), v)
            return out.index_add(0, torch.as_tensor(bj), v)

        del ones_b
        val = _t(P["val"][ty])
        dp = atom_sum(bop) - val                                  # Delta'
        dpboc = atom_sum(bop) - _t(P["valboc"][ty])               # Delta'boc
        pb1, pb2 = P["p_boc1"], P["p_boc2"]
        dpi, dpj = dp[bi], dp[bj]
        f2 = torch.exp(-pb1 * dpi) + torch.exp(-pb1 * dpj)
        f3 = -(1.0 / pb2) * torch.log(0.5 * (torch.exp(-pb2 * dpi) + torch.exp(-pb2 * dpj)))
        vi, vj = val[bi], val[bj]
        f1 = 0.5 * ((vi + f2) / (vi + f2 + f3) + (vj + f2) / (vj + f2 + f3))
        ovc = _t(P["ovc"][ti, tj])
        f1 = torch.where(ovc > 0, f1, torch.ones_like(f1))
        p3, p4, p5 = _t(P["p_boc3"][ti, tj]), _t(P["p_boc4"][ti, tj]), _t(P["p_boc5"][ti, tj])
        f4 = _sig(-p3 * (p4 * bop * bop - dpboc[bi]) + p5)
        f5 = _sig(-p3 * (p4 * bop * bop - dpboc[bj]) + p5)
        v13 = _t(P["v13"][ti, tj])
        f4 = torch.where(v13 > 0, f4, torch.ones_like(f4))
        f5 = torch.where(v13 > 0, f5, torch.ones_like(f5))
        BO = bop * f1 * f4 * f5
        BOpi = bp * f1 * f1 * f4 * f5
        BOpp = bpp * f1 * f1 * f4 * f5
        BOs = BO - BOpi - BOpp
        parts.update(bo_prime=bop.detach().numpy(), bo=BO.detach().numpy(),
                     bo_pi=BOpi.detach().numpy(), bo_pp=BOpp.detach().numpy(),
                     f1=f1.detach().numpy(), f4=f4.detach().numpy(), f5=f5.detach().numpy())

        # ---------------- atom quantities
        sumBO = atom_sum(BO)
        Delta = sumBO - val
        Dele = sumBO - _t(P["vale"][ty])
        Dang = sumBO - _t(P["valang"][ty])
        Tr = torch.trunc(Dele.detach() / 2.0)                       # constant in derivatives
        el = 2.0 + Dele - 2.0 * Tr
        nlp = torch.exp(-P["p_lp1"] * el * el) - Tr
        nlp_opt = 0.5 * (_t(P["vale"][ty]) - val)
        Dlp = nlp_opt - nlp
        parts.update(delta=Delta.detach().numpy(), nlp=nlp.detach().numpy(), dlp=Dlp.detach().numpy(),
                     sumbo=sumBO.detach().numpy())

        def tot(name, e):
            if name in mask:
                E[name] = e.sum()
            else:
                E[name] = (e * 0.0).sum()

        # ---------------- bond energy
        dsg = _t(P["De_s"][ti, tj])
        pbe1, pbe2 = _t(P["p_be1"][ti, tj]), _t(P["p_be2"][ti, tj])
        pos = BOs > 0
        bsafe = torch.where(pos, BOs, torch.ones_like(BOs))
        esig = -dsg * bsafe * torch.exp(pbe1 * (1.0 - torch.pow(bsafe, pbe2)))
        esig = torch.where(pos, esig, torch.zeros_like(esig))
        tot("bond", esig - _t(P["De_p"][ti, tj]) * BOpi - _t(P["De_pp"][ti, tj]) * BOpp)

        # ---------------- lone pair, over- and under-coordination
        elp = _t(P["p_lp2"][ty]) * Dlp * torch.sigmoid(75.0 * Dlp)
        tot("lp", elp)
        dd = (Delta - Dlp)
        S = torch.zeros(n, dtype=_DT)
        S = S.index_add(0, torch.as_tensor(bi), dd[bj] * (BOpi + BOpp))
        S = S.index_add(0, torch.as_tensor(bj), dd[bi] * (BOpi + BOpp))
        Dlpc = Delta - Dlp / (1.0 + P["p_ovun3"] * torch.exp(P["p_ovun4"] * S))
        sov = atom_sum(_t(P["p_ovun1"][ti, tj]) * dsg * BO)
        pov2 = _t(P["p_ovun2"][ty])
        eov = sov * Dlpc / (Dlpc + val + 1e-8) * _sig(pov2 * Dlpc)
        tot("over", eov)
        eun = -_t(P["p_ovun5"][ty]) * (1.0 - torch.exp(P["p_ovun6"] * Dlpc)) * _sig(-pov2 * Dlpc) \
            / (1.0 + P["p_ovun7"] * torch.exp(P["p_ovun8"] * S))
        tot("under", eun)
        parts.update(S=S.detach().numpy(), dlpc=Dlpc.detach().numpy())

        # ---------------- valence angle, penalty, coalition (centre j)
        D = L.get("_directed")
        if D is None:
            D = L["_directed"] = _directed(B, n)
        bo_np = BO.detach().numpy()
        ea, eb = L.get("_angles", (None, None))
        if ea is None:
            ea, eb = enumerate_angles(D, n)
            L["_angles"] = (ea, eb)
        b1, b2 = D["b"][ea], D["b"][eb]
        BO1, BO2 = bo_np[b1], bo_np[b2]
        keep = (BO1 > o["thb_cut"]) & (BO2 > o["thb_cut"]) & (BO1 * BO2 > o["thb_cutsq"])
        ea, eb = ea[keep], eb[keep]
        jj = D["c"][ea]
        ii, kk = D["o"][ea], D["o"][eb]
        b1, b2 = D["b"][ea], D["b"][eb]
        sg1, sg2 = _t(D["sg"][ea])[:, None], _t(D["sg"][eb])[:, None]
        v1 = db[b1] * sg1                             # j -> i
        v2 = db[b2] * sg2                             # j -> k
        r1 = torch.sqrt((v1 * v1).sum(1))
        r2 = torch.sqrt((v2 * v2).sum(1))
        cth = torch.clamp((v1 * v2).sum(1) / (r1 * r2), -1.0, 1.0)
        th = torch.acos(cth)
        BOa, BOb = BO[b1], BO[b2]
        # SBO of centre j
        pisum = atom_sum(BOpi + BOpp)
        prod = torch.exp(-atom_sum(BO ** 8))
        SBO = pisum + (1.0 - prod) * (-Dang - P["p_val8"] * nlp)
        p9 = P["p_val9"]
        s_lo = torch.clamp(SBO, 1e-30, 1.0)
        s_hi = torch.clamp(2.0 - SBO, 1e-30, 1.0)
        SBO2 = torch.where(SBO <= 0, torch.zeros_like(SBO),
                           torch.where(SBO < 1, torch.pow(s_lo, p9),
                                       torch.where(SBO < 2, 2.0 - torch.pow(s_hi, p9), 2.0 * torch.ones_like(SBO))))
        tj_, ti_, tk_ = ty[jj], ty[ii], ty[kk]
        th0 = math.pi - _t(P["th00"][ti_, tj_, tk_]) * (1.0 - torch.exp(-P["p_val10"] * (2.0 - SBO2[jj])))
        pv3 = _t(P["p_val3"][tj_])
        pv4 = _t(P["p_val4"][ti_, tj_, tk_])
        f7a = 1.0 - torch.exp(-pv3 * torch.pow(BOa, pv4))
        f7b = 1.0 - torch.exp(-pv3 * torch.pow(BOb, pv4))
        pv5 = _t(P["p_val5"][tj_])
        Dj = Dang[jj]
        e6 = torch.exp(P["p_val6"] * Dj)
        f8 = pv5 - (pv5 - 1.0) * (2.0 + e6) / (1.0 + e6 + torch.exp(-_t(P["p_val7"][ti_, tj_, tk_]) * Dj))
        eval_ = f7a * f7b * f8 * _t(P["p_val1"][ti_, tj_, tk_]) * \
            (1.0 - torch.exp(-_t(P["p_val2"][ti_, tj_, tk_]) * (th0 - th) ** 2))
        tot("val", eval_)
        Dd = Delta[jj]
        f9 = (2.0 + torch.exp(-P["p_pen3"] * Dd)) / (1.0 + torch.exp(-P["p_pen3"] * Dd) + torch.exp(P["p_pen4"] * Dd))
        epen = _t(P["p_pen1"][ti_, tj_, tk_]) * f9 * torch.exp(-P["p_pen2"] * (BOa - 2.0) ** 2) \
            * torch.exp(-P["p_pen2"] * (BOb - 2.0) ** 2)
        tot("pen", epen)
        ecoa = _t(P["p_coa1"][ti_, tj_, tk_]) * _sig(P["p_coa2"] * Dj) \
            * torch.exp(-P["p_coa3"] * (sumBO[ii] - BOa) ** 2) * torch.exp(-P["p_coa3"] * (sumBO[kk] - BOb) ** 2) \
            * torch.exp(-P["p_coa4"] * (BOa - 1.5) ** 2) * torch.exp(-P["p_coa4"] * (BOb - 1.5) ** 2)
        tot("coa", ecoa)
        parts.update(n_angles=int(len(ea)), sbo=SBO.detach().numpy())

        # ---------------- torsion and conjugation (central bond j-k)
        tA = L.get("_tors")
        if tA is None:
            tA = L["_tors"] = enumerate_torsions(D, B, n)
        ea4, ec4, bc = tA
        # geometry of the point l relative to j must differ from i's
        sh_i = D["sh"][ea4]                                  # i relative to j
        sh_l = B["s"][bc] + D["sh"][ec4]                      # l relative to j
        same_pt = (D["o"][ea4] == D["o"][ec4]) & np.all(sh_i == sh_l, axis=1)
        BOij, BOjk, BOkl = bo_np[D["b"][ea4]], bo_np[bc], bo_np[D["b"][ec4]]
        keep = (~same_pt) & (BOjk > o["thb_cut"]) & (BOij * BOjk * BOkl > o["thb_cut"])
        ea4, ec4, bc = ea4[keep], ec4[keep], bc[keep]
        jj4, kk4 = B["i"][bc], B["j"][bc]
        u1 = db[D["b"][ea4]] * _t(D["sg"][ea4])[:, None]     # j -> i
        u2 = db[bc]                                           # j -> k
        u3 = db[D["b"][ec4]] * _t(D["sg"][ec4])[:, None]     # k -> l
        l1 = torch.sqrt((u1 * u1).sum(1))
        l2 = torch.sqrt((u2 * u2).sum(1))
        l3 = torch.sqrt((u3 * u3).sum(1))
        c1 = torch.clamp((u1 * u2).sum(1) / (l1 * l2), -1.0, 1.0)
        c2 = torch.clamp(-(u2 * u3).sum(1) / (l2 * l3), -1.0, 1.0)
        s1 = torch.clamp(torch.sqrt(torch.clamp(1.0 - c1 * c1, min=0.0)), min=1e-10)
        s2 = torch.clamp(torch.sqrt(torch.clamp(1.0 - c2 * c2, min=0.0)), min=1e-10)
        # (u1 x u2) . ((-u2) x u3) = (u1.u3)|u2|^2 - (u1.u2)(u2.u3)
        Pn = (u1 * u3).sum(1) * (l2 * l2) - (u1 * u2).sum(1) * (u2 * u3).sum(1)
        cw = torch.clamp(Pn / (l1 * l2 * l2 * l3 * s1 * s2), -1.0, 1.0)
        tj4, tk4 = ty[jj4], ty[kk4]
        BO1, BO2, BO3 = BO[D["b"][ea4]], BO[bc], BO[D["b"][ec4]]
        pt2 = P["p_tor2"]
        f10 = (1.0 - torch.exp(-pt2 * BO1)) * (1.0 - torch.exp(-pt2 * BO2)) * (1.0 - torch.exp(-pt2 * BO3))
        Dsum = Dang[jj4] + Dang[kk4]
        f11 = (2.0 + torch.exp(-P["p_tor3"] * Dsum)) / (1.0 + torch.exp(-P["p_tor3"] * Dsum) + torch.exp(P["p_tor4"] * Dsum))
        V1, V2, V3 = _t(P["V1"][tj4, tk4]), _t(P["V2"][tj4, tk4]), _t(P["V3"][tj4, tk4])
        pt1 = _t(P["p_tor1"][tj4, tk4])
        c2w = 2.0 * cw * cw - 1.0
        c3w = 4.0 * cw * cw * cw - 3.0 * cw
        etor = f10 * s1 * s2 * (0.5 * V1 * (1.0 + cw)
                                + 0.5 * V2 * torch.exp(pt1 * (2.0 - BOpi[bc] - f11) ** 2) * (1.0 - c2w)
                                + 0.5 * V3 * (1.0 + c3w))
        tot("tors", etor)
        pc2 = P["p_cot2"]
        econ = _t(P["p_cot1"][tj4, tk4]) * torch.exp(-pc2 * (BO1 - 1.5) ** 2) * torch.exp(-pc2 * (BO2 - 1.5) ** 2) \
            * torch.exp(-pc2 * (BO3 - 1.5) ** 2) * (1.0 + (cw * cw - 1.0) * s1 * s2)
        tot("conj", econ)
        parts.update(n_torsions=int(len(bc)))

        # ---------------- hydrogen bonds (H atom j, bonded X = i, partner Z = k)
        HB = L["hbond"]
        hbf = P["hb"]
        # bonded X of each H: directed entries with centre H, other flag 2, BO >= hb_bo_min
        ent = np.nonzero((hbf[ty[D["c"]]] == 1) & (hbf[ty[D["o"]]] == 2) & (bo_np[D["b"]] >= o["hb_bo_min"]))[0]
        hstart = np.searchsorted(HB["i"], np.arange(n + 1)) if len(HB["i"]) else np.zeros(n + 1, np.int64)
        if len(HB["i"]):
            assert np.all(np.diff(HB["i"]) >= 0)
        cnt = hstart[D["c"][ent] + 1] - hstart[D["c"][ent]]
        e_rep = np.repeat(ent, cnt)
        off = np.repeat(np.cumsum(cnt) - cnt, cnt)
        zi = np.repeat(hstart[D["c"][ent]], cnt) + (np.arange(int(cnt.sum())) - off)
        same = (HB["j"][zi] == D["o"][e_rep]) & np.all(HB["s"][zi] == D["sh"][e_rep], axis=1)
        e_rep, zi = e_rep[~same], zi[~same]
        hj = D["c"][e_rep]
        hx = D["o"][e_rep]
        hz = HB["j"][zi]
        w1 = db[D["b"][e_rep]] * _t(D["sg"][e_rep])[:, None]     # H -> X
        w2 = dvec(HB["i"][zi], hz, HB["s"][zi])                  # H -> Z
        q1 = torch.sqrt((w1 * w1).sum(1))
        q2 = torch.sqrt((w2 * w2).sum(1))
        ch = torch.clamp((w1 * w2).sum(1) / (q1 * q2), -1.0, 1.0)
        tx, tz = ty[hx], ty[hz]
        r0h = _t(P["r0hb"][tx, tz])
        ehb = _t(P["p_hb1"][tx, tz]) * (1.0 - torch.exp(-_t(P["p_hb2"][tx, tz]) * BO[D["b"][e_rep]])) \
            * torch.exp(-_t(P["p_hb3"][tx, tz]) * (r0h / q2 + q2 / r0h - 2.0)) * (0.5 * (1.0 - ch)) ** 2
        tot("hbond", ehb)
        parts.update(n_hbonds=int(len(zi)))
        del hj

        # ---------------- van der Waals and Coulomb over the canonical half far list
        Fl = L["far"]
        hm = half_mask(Fl["i"], Fl["j"], Fl["s"])
        pi_, pj_ = Fl["i"][hm], Fl["j"][hm]
        dn = dvec(pi_, pj_, Fl["s"][hm])
        rn = torch.sqrt((dn * dn).sum(1))
        tap = taper(rn, o["r_nb"])
        a_, b_ = ty[pi_], ty[pj_]
        pv = P["p_vdW1"]
        f13 = torch.pow(torch.pow(rn, pv) + _t(P["vdw_gw"][a_, b_]) ** (-pv), 1.0 / pv)
        al = _t(P["vdw_alpha"][a_, b_])
        xr = 1.0 - f13 / _t(P["vdw_rv"][a_, b_])
        evdw = tap * _t(P["vdw_D"][a_, b_]) * (torch.exp(al * xr) - 2.0 * torch.exp(0.5 * al * xr))
        tot("vdw", evdw)
        qq = _t(q)
        g = _t(P["gamma"][a_, b_])
        ecoul = tap * P["k_e"] * qq[pi_] * qq[pj_] / torch.pow(rn ** 3 + g ** -3.0, 1.0 / 3.0)
        tot("coul", ecoul)
        epol = _t(P["chi"][ty]) * qq + 0.5 * _t(P["eta"][ty]) * qq * qq
        tot("pol", epol)

        Etot = sum(E.values())
        out = dict(E={k: float(v.detach()) for k, v in E.items()}, parts=parts)
        out["E_total"] = float(Etot.detach())
        if need_grad:
            gx, ge = torch.autograd.grad(Etot, (X, EPS), allow_unused=True)
            out["F"] = (-gx).numpy() if gx is not None else np.zeros((n, 3))
            out["W"] = (-ge).numpy() if ge is not None else np.zeros((3, 3))
        return out

    # ---------------------------------------------------------------- one MD step
    def forces(self, x, q=None, tol=None, guess=None, term_mask=None, brute=None):
        """Lists, QEq (unless q is given), energy terms, forces and virial at x."""
        L = self.lists(x, brute=brute)
        qq = self.qeq(x, L, tol=tol, guess=guess) if q is None else dict(q=np.asarray(q, float))
        out = self.energy(x, qq["q"], L, term_mask=self.term_mask if term_mask is None else term_mask)
        out["qeq"] = qq
        out["lists"] = L
        return out


def pcg(Hm, b, diag, tol, max_iter, x0=None):
    """Jacobi-preconditioned conjugate gradient (M = diag(H)) for H x = b.
    Stops when ||r||_2 / ||b||_2 <= tol; returns (x, iterations)."""
    x = np.zeros_like(b) if x0 is None else np.array(x0, float)
    r = b - Hm @ x
    bn = np.linalg.norm(b)
    if np.linalg.norm(r) <= tol * bn:
        return x, 0
    z = r / diag
    p = z.copy()
    rz = r @ z
    for it in range(1, max_iter + 1):
        w = Hm @ p
        alpha = rz / (p @ w)
        x = x + alpha * p
        r = r - alpha * w
        if np.linalg.norm(r) <= tol * bn:
            return x, it
        z = r / diag
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, max_iter


def blocks_of(rep_offsets, size=32):
    """Blocks of `size` consecutive atoms of each replica (the last block of a replica may be
    shorter): list of (start, stop)."""
    out = []
    for r in range(len(rep_offsets) - 1):
        for a in range(rep_offsets[r], rep_offsets[r + 1], size):
            out.append((a, min(a + size, rep_offsets[r + 1])))
    return out


def pcg_block(Hm, b, blocks, tol, max_iter, x0=None):
    """Block-Jacobi preconditioned CG for H x = b: M = blockdiag(H_BB) over the given
    blocks (each H_BB the restriction of H to the block, every entry of H kept), applied as
    z = H_BB^-1 r per block (dense FP64 inverse). Same stopping rule as pcg(): the
    iteration ends when ||r||_2 / ||b||_2 <= tol. Returns (x, iterations)."""
    Hd = Hm.tocsr()
    inv = [(a, e, np.linalg.inv(Hd[a:e, a:e].toarray())) for a, e in blocks]

    def apply(r):
        z = np.empty_like(r)
        for a, e, Bi in inv:
            z[a:e] = Bi @ r[a:e]
        return z

    x = np.zeros_like(b) if x0 is None else np.array(x0, float)
    r = b - Hm @ x
    bn = np.linalg.norm(b)
    if np.linalg.norm(r) <= tol * bn:
        return x, 0
    z = apply(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, max_iter + 1):
        w = Hm @ p
        alpha = rz / (p @ w)
        x = x + alpha * p
        r = r - alpha * w
        if np.linalg.norm(r) <= tol * bn:
            return x, it
        z = apply(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, max_iter


def gmres(Hm, b, diag, tol, max_iter, restart=50, x0=None):
    """Restarted GMRES(m) for H x = b (Saad and Schultz), right Jacobi preconditioning
    (H M^-1 y = b, x = M^-1 y, M = diag), Arnoldi by modified Gram-Schmidt, the small least-
    squares problem by Givens rotations. Same stopping rule as pcg(): ||r||_2 / ||b||_2 <=
    tol. Returns (x, iterations, residual-norm history). Sec. 3.3 names GMRES beside CG for
    the QEq systems; this is the solver-variant comparison, not the path's solver."""
    n = len(b)
    x = np.zeros(n) if x0 is None else np.array(x0, float)
    bn = np.linalg.norm(b)
    r = b - Hm @ x
    beta = np.linalg.norm(r)
    hist = [beta / bn]
    it = 0
    while beta > tol * bn and it < max_iter:
        m = min(restart, max_iter - it)
        V = np.zeros((m + 1, n))
        Hh = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k_used = 0
        for k in range(m):
            w = Hm @ (V[k] / diag)
            for jj in range(k + 1):
                Hh[jj, k] = w @ V[jj]
                w = w - Hh[jj, k] * V[jj]
            Hh[k + 1, k] = np.linalg.norm(w)
            if Hh[k + 1, k] > 0:
                V[k + 1] = w / Hh[k + 1, k]
            for jj in range(k):                        # earlier rotations on the new column
                t = cs[jj] * Hh[jj, k] + sn[jj] * Hh[jj + 1, k]
                Hh[jj + 1, k] = -sn[jj] * Hh[jj, k] + cs[jj] * Hh[jj + 1, k]
                Hh[jj, k] = t
            den = np.hypot(Hh[k, k], Hh[k + 1, k])
            cs[k], sn[k] = Hh[k, k] / den, Hh[k + 1, k] / den
            Hh[k, k] = den
            Hh[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            it += 1
            k_used = k + 1
            hist.append(abs(g[k + 1]) / bn)
            if abs(g[k + 1]) <= tol * bn:
                break
        y = np.linalg.solve(np.triu(Hh[:k_used, :k_used]), g[:k_used])
        x = x + (V[:k_used].T @ y) / diag
        r = b - Hm @ x
        beta = np.linalg.norm(r)
    return x, it, np.array(hist)


def kinetic(v, masses):
    """Kinetic energy (kcal/mol) of velocities in A/fs."""
    return 0.5 * float((masses[:, None] * v * v).sum()) / ACC_CONV


def free_flight(x, v, box, dt, nsteps):
    """Velocity Verlet with every force zero: the velocities stay, and each step moves
    x to x + dt v (product and sum rounded separately) and wraps it into the box."""
    x = np.array(x, float)
    v = np.asarray(v, float)
    box = np.asarray(box, float)
    for _ in range(nsteps):
        x = x + dt * v
        x = np.where(x < 0, x + box, x)
        x = np.where(x >= box, x - box, x)
    return x


def verlet(model, x, v, dt, nsteps, F=None, q_hist=None):
    """Velocity Verlet (dt in fs): v += dt/2 a; x += dt v (wrapped into the box);
    recompute forces; v += dt/2 a. Returns x, v, F and per-step total energy."""
    m = model.P["mass"][model.types]
    box = model.box
    if F is None:
        F = model.forces(x)["F"]
    etot = []
    for _ in range(nsteps):
        v = v + 0.5 * dt * ACC_CONV * F / m[:, None]
        x = x + dt * v
        x = np.where(x < 0, x + box, x)
        x = np.where(x >= box, x - box, x)
        out = model.forces(x)
        F = out["F"]
        v = v + 0.5 * dt * ACC_CONV * F / m[:, None]
        etot.append(out["E_total"] + kinetic(v, m))
    return x, v, F, np.array(etot)
