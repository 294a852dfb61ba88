"""Python binding of libreaxff.so (include/reaxff.h): argument marshalling only.

Every computation runs in the library's CUDA kernels. The module-level functions carry
the C names; `ReaxFF` wraps one context. Loading fails loudly when the library is
missing (build it with `python -m paper_1706_07772_gb300.build`).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

MAXT = 8
NTERMS = 13
TERMS = ("bond", "lp", "over", "under", "val", "pen", "coa", "tors", "conj", "hbond", "vdw", "coul", "pol")
NO_TERMS = 1 << NTERMS     # term mask that selects no term: zero forces (free flight)
OK, E_INVALID, E_CUDA, E_CAPACITY, E_NOT_CONVERGED, E_TIMEOUT, E_NAN, E_STATE = 0, -1, -2, -3, -4, -5, -6, -7
FP64, MIXED = 0, 1
WARM_EXTRAP, WARM_ZERO, WARM_MLP, WARM_LAGRANGE = 0, 1, 2, 3
PRECOND_JACOBI, PRECOND_BLOCK32 = 0, 1
LIST_FAR, LIST_BOND, LIST_HBOND = 0, 1, 2

_PER_TYPE = ("mass", "val", "vale", "valboc", "valang", "p_lp2", "p_ovun2", "p_ovun5", "p_val3", "p_val5",
             "chi", "eta", "gamma_t")
_PER_PAIR = ("r0s", "r0p", "r0pp", "p_bo1", "p_bo2", "p_bo3", "p_bo4", "p_bo5", "p_bo6", "p_boc3", "p_boc4",
             "p_boc5", "ovc", "v13", "De_s", "De_p", "De_pp", "p_be1", "p_be2", "p_ovun1", "vdw_D", "vdw_rv",
             "vdw_alpha", "vdw_gw", "gamma")
_PER_TRIPLE = ("th00", "p_val1", "p_val2", "p_val4", "p_val7", "p_pen1", "p_coa1")
_PER_PAIR2 = ("V1", "V2", "V3", "p_tor1", "p_cot1", "r0hb", "p_hb1", "p_hb2", "p_hb3")
_GENERAL = ("p_boc1", "p_boc2", "p_lp1", "p_ovun3", "p_ovun4", "p_ovun6", "p_ovun7", "p_ovun8", "p_val6",
            "p_val8", "p_val9", "p_val10", "p_pen2", "p_pen3", "p_pen4", "p_coa2", "p_coa3", "p_coa4",
            "p_tor2", "p_tor3", "p_tor4", "p_cot2", "p_vdW1", "k_e")

_D8 = C.c_double * MAXT
_D88 = _D8 * MAXT
_D888 = _D88 * MAXT


class Params(C.Structure):
    _fields_ = ([("ntypes", C.c_int32), ("hb", C.c_int32 * MAXT)] + [(k, _D8) for k in _PER_TYPE]
                + [(k, _D88) for k in _PER_PAIR] + [(k, _D888) for k in _PER_TRIPLE]
                + [(k, _D88) for k in _PER_PAIR2] + [(k, C.c_double) for k in _GENERAL])


class Options(C.Structure):
    _fields_ = [("r_nb", C.c_double), ("r_bond", C.c_double), ("r_hb", C.c_double), ("bo_cut", C.c_double),
                ("thb_cut", C.c_double), ("thb_cutsq", C.c_double), ("hb_bo_min", C.c_double),
                ("qeq_tol", C.c_double), ("qeq_max_iter", C.c_int32), ("precision", C.c_int32),
                ("warm_start", C.c_int32), ("term_mask", C.c_int32), ("capacity_margin", C.c_double),
                ("skin", C.c_double), ("qeq_precond", C.c_int32), ("spatial_sort", C.c_int32)]


class ReaxFFError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("reaxff error %d: %s" % (code, msg))
        self.code = code


LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libreaxff.so")
_lib = None


def load(path: str = LIB_PATH):
    """Load libreaxff.so and check the struct layouts against the library's own."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libreaxff.so not built: run `python -m paper_1706_07772_gb300.build` (%s)" % path)
    lib = C.CDLL(path)
    vp, i32, i64, dp, ip32, ip64 = C.c_void_p, C.c_int32, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_int64)
    fp = C.POINTER(C.c_float)
    sig = {
        "reaxff_sizeof_params": (i64, []), "reaxff_sizeof_options": (i64, []),
        "reaxff_params_offset": (i64, [C.c_char_p]),
        "reaxff_create": (C.c_int, [C.POINTER(Params), ip32, i64, dp, C.POINTER(Options), C.POINTER(vp)]),
        "reaxff_create_batch": (C.c_int, [C.POINTER(Params), i32, ip64, ip32, dp, C.POINTER(Options), C.POINTER(vp)]),
        "reaxff_destroy": (None, [vp]), "reaxff_last_error": (C.c_char_p, [vp]),
        "reaxff_num_atoms": (i64, [vp]), "reaxff_num_replicas": (i32, [vp]),
        "reaxff_set_state": (C.c_int, [vp, dp, dp]), "reaxff_get_state": (C.c_int, [vp, dp, dp, dp]),
        "reaxff_resort": (C.c_int, [vp]),
        "reaxff_build_lists": (C.c_int, [vp]),
        "reaxff_get_lists": (C.c_int, [vp, i32, i64, ip64, ip32, ip32, C.POINTER(C.c_int8)]),
        "reaxff_get_bond_orders": (C.c_int, [vp, i64, ip64, dp, dp, dp, dp]),
        "reaxff_qeq": (C.c_int, [vp, dp, ip32, ip32]),
        "reaxff_forces": (C.c_int, [vp, dp, dp, dp]),
        "reaxff_forces_fixed_q": (C.c_int, [vp, dp, dp, dp, dp]),
        "reaxff_step": (C.c_int, [vp, i32, C.c_double, dp]),
        "reaxff_last_launch_count": (i64, [vp]),
        "reaxff_set_state_dev": (C.c_int, [vp, vp, vp, vp]),
        "reaxff_get_state_dev": (C.c_int, [vp, vp, vp, vp, vp]),
        "reaxff_step_dev": (C.c_int, [vp, i32, C.c_double, vp, vp]),
        "reaxff_reset_qeq_history": (None, [vp]),
        "reaxff_set_wait_limit": (C.c_int, [vp, i64]),
        "reaxff_qeq_spmv_total": (i64, [vp]),
        "reaxff_qeq_warm_choice": (C.c_int, [vp, ip32]),
        "reaxff_species": (C.c_int, [vp, dp, ip32, ip64, i32, ip32, ip32]),
        "reaxff_species_average": (C.c_int, [vp, dp, ip32, ip64, i32, ip32, ip32]),
        "reaxff_bo_average_reset": (C.c_int, [vp]), "reaxff_bo_average_sample": (C.c_int, [vp]),
        "reaxff_bo_average_samples": (i64, [vp]),
        "reaxff_get_bo_average": (C.c_int, [vp, i64, ip64, ip32, ip32, C.POINTER(C.c_int8), dp]),
        "reaxff_autotune": (C.c_int, [vp, C.c_char_p, ip32]),
        "reaxff_extrap_weights": (C.c_int, [i32, dp]),
        "reaxff_mlp_init": (C.c_int, [vp, C.c_uint64]),
        "reaxff_mlp_set_params": (C.c_int, [vp, fp, fp, fp]),
        "reaxff_mlp_get_params": (C.c_int, [vp, fp, fp, fp]),
        "reaxff_mlp_descriptors": (C.c_int, [vp, fp]),
        "reaxff_mlp_infer": (C.c_int, [vp, fp, ip32, i64, fp]),
        "reaxff_mlp_loss_grad": (C.c_int, [vp, fp, ip32, fp, i64, fp, dp]),
        "reaxff_mlp_adam_step": (C.c_int, [vp, fp, C.c_double]),
        "reaxff_mlp_reserve": (C.c_int, [vp, i32]),
        "reaxff_mlp_collect": (C.c_int, [vp]),
        "reaxff_mlp_train": (C.c_int, [vp, i32, C.c_double, dp]),
        "reaxff_mlp_predict": (C.c_int, [vp, dp]),
        "reaxff_last_qeq_iters": (C.c_int, [vp, ip32, ip32]),
        "reaxff_profile_enable": (None, [vp, i32]),
        "reaxff_profile_read": (i32, [vp, i32, dp, ip64]),
        "reaxff_stage_name": (C.c_char_p, [i32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if lib.reaxff_sizeof_params() != C.sizeof(Params) or lib.reaxff_sizeof_options() != C.sizeof(Options):
        raise ImportError("reaxff struct size mismatch between binding and library")
    for name, _ in Params._fields_:
        if lib.reaxff_params_offset(name.encode()) != getattr(Params, name).offset:
            raise ImportError("reaxff_params field offset mismatch: " + name)
    _lib = lib
    return lib


def _fp(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def make_params(p: dict) -> Params:
    """Pack a parameter dict (numpy tables, types 0..ntypes-1) into the C struct."""
    P = Params()
    nt = int(p["ntypes"])
    P.ntypes = nt
    for t in range(nt):
        P.hb[t] = int(p["hb"][t])
    for k in _PER_TYPE:
        arr = getattr(P, k)
        for t in range(nt):
            arr[t] = float(p[k][t])
    for k in _PER_PAIR + _PER_PAIR2:
        arr = getattr(P, k)
        v = np.asarray(p[k], float)
        for a in range(nt):
            for b in range(nt):
                arr[a][b] = v[a, b]
    for k in _PER_TRIPLE:
        arr = getattr(P, k)
        v = np.asarray(p[k], float)
        for a in range(nt):
            for b in range(nt):
                for c in range(nt):
                    arr[a][b][c] = v[a, b, c]
    for k in _GENERAL:
        setattr(P, k, float(p[k]))
    return P


def make_options(o: dict, precision=FP64, warm_start=WARM_EXTRAP, term_mask=0, capacity_margin=0.0,
                 skin=0.0, qeq_precond=0, spatial_sort=0) -> Options:
    O = Options()
    for k in ("r_nb", "r_bond", "r_hb", "bo_cut", "thb_cut", "thb_cutsq", "hb_bo_min", "qeq_tol"):
        setattr(O, k, float(o[k]))
    O.qeq_max_iter = int(o.get("qeq_max_iter", 200))
    O.precision = int(precision)
    O.warm_start = int(warm_start)
    O.term_mask = int(term_mask)
    O.capacity_margin = float(capacity_margin)
    O.skin = float(o.get("skin", skin))
    O.qeq_precond = int(o.get("qeq_precond", qeq_precond))
    O.spatial_sort = int(o.get("spatial_sort", spatial_sort))
    return O


def extrap_weights(predictor=0):
    """Weights w[sys, m, k] of initial-guess predictor 0 (Lagrange), 1 or 2 (least squares
    over 6 or 8 solutions); host only."""
    w = np.empty(2 * 9 * 8)
    rc = load().reaxff_extrap_weights(int(predictor), _dp(w))
    if rc != OK:
        raise ReaxFFError(rc, "reaxff_extrap_weights failed")
    return w.reshape(2, 9, 8)


def term_mask(*names) -> int:
    m = 0
    for nm in names:
        m |= 1 << TERMS.index(nm)
    return m


# ------------------------------------------------------------------ C-named wrappers
def reaxff_create(params: Params, types, box, options: Options):
    lib = load()
    t = np.ascontiguousarray(types, np.int32)
    b = np.ascontiguousarray(box, np.float64)
    h = C.c_void_p()
    rc = lib.reaxff_create(C.byref(params), t.ctypes.data_as(C.POINTER(C.c_int32)), len(t), _dp(b),
                           C.byref(options), C.byref(h))
    if rc != OK:
        raise ReaxFFError(rc, "reaxff_create failed")
    return h


def reaxff_create_batch(params: Params, rep_offsets, types, boxes, options: Options):
    lib = load()
    off = np.ascontiguousarray(rep_offsets, np.int64)
    t = np.ascontiguousarray(types, np.int32)
    b = np.ascontiguousarray(boxes, np.float64).reshape(-1)
    h = C.c_void_p()
    rc = lib.reaxff_create_batch(C.byref(params), len(off) - 1, off.ctypes.data_as(C.POINTER(C.c_int64)),
                                 t.ctypes.data_as(C.POINTER(C.c_int32)), _dp(b), C.byref(options), C.byref(h))
    if rc != OK:
        raise ReaxFFError(rc, "reaxff_create_batch failed")
    return h


class ReaxFF:
    """One library context (single system or a batch of replicas)."""

    def __init__(self, params: dict, types, box, options: dict, precision=FP64, warm_start=WARM_EXTRAP,
                 term_mask=0, rep_offsets=None, capacity_margin=0.0, skin=0.0, qeq_precond=0, spatial_sort=0):
        self.lib = load()
        P = make_params(params)
        O = make_options(options, precision, warm_start, term_mask, capacity_margin, skin, qeq_precond,
                         spatial_sort)
        self.types = np.ascontiguousarray(types, np.int32)
        if rep_offsets is None:
            self.h = reaxff_create(P, self.types, np.asarray(box, float).reshape(3), O)
        else:
            self.h = reaxff_create_batch(P, rep_offsets, self.types, np.asarray(box, float), O)
        self.n = int(self.lib.reaxff_num_atoms(self.h))
        self.nrep = int(self.lib.reaxff_num_replicas(self.h))

    def _check(self, rc, allow=()):
        if rc != OK and rc not in allow:
            raise ReaxFFError(rc, self.lib.reaxff_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.lib.reaxff_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, x, v=None):
        x = np.ascontiguousarray(x, np.float64).reshape(self.n, 3)
        v = None if v is None else np.ascontiguousarray(v, np.float64).reshape(self.n, 3)
        self._check(self.lib.reaxff_set_state(self.h, _dp(x), _dp(v)))

    def resort(self):
        """Store the atoms again in cell order of their current positions (spatial_sort)."""
        self._check(self.lib.reaxff_resort(self.h))

    def get_state(self, out=None):
        """Positions, velocities and charges; `out` = (x, v, q) C-contiguous float64 arrays
        of shapes (n, 3), (n, 3), (n,) to fill instead of new ones (e.g. pinned buffers)."""
        if out is None:
            x = np.empty((self.n, 3))
            v = np.empty((self.n, 3))
            q = np.empty(self.n)
        else:
            x, v, q = out
            for a, shape in ((x, (self.n, 3)), (v, (self.n, 3)), (q, (self.n,))):
                if a.shape != shape or a.dtype != np.float64 or not a.flags.c_contiguous:
                    raise ValueError("get_state out arrays must be C-contiguous float64 of shape %s" % (shape,))
        self._check(self.lib.reaxff_get_state(self.h, _dp(x), _dp(v), _dp(q)))
        return x, v, q

    def build_lists(self):
        self._check(self.lib.reaxff_build_lists(self.h))

    def list_count(self, which):
        """Entries of a list (both directions for the far and bond lists)."""
        cnt = C.c_int64()
        self._check(self.lib.reaxff_get_lists(self.h, which, 0, C.byref(cnt), None, None, None))
        return cnt.value

    def get_lists(self, which):
        cnt = C.c_int64()
        self._check(self.lib.reaxff_get_lists(self.h, which, 0, C.byref(cnt), None, None, None))
        m = cnt.value
        i = np.empty(m, np.int32)
        j = np.empty(m, np.int32)
        s = np.empty((m, 3), np.int8)
        self._check(self.lib.reaxff_get_lists(self.h, which, m, C.byref(cnt), i.ctypes.data_as(C.POINTER(C.c_int32)),
                                              j.ctypes.data_as(C.POINTER(C.c_int32)),
                                              s.ctypes.data_as(C.POINTER(C.c_int8))))
        return i, j, s

    def get_bond_orders(self):
        cnt = C.c_int64()
        self._check(self.lib.reaxff_get_bond_orders(self.h, 0, C.byref(cnt), None, None, None, None))
        m = cnt.value
        out = {k: np.empty(m) for k in ("bo_prime", "bo", "bo_pi", "bo_pp")}
        self._check(self.lib.reaxff_get_bond_orders(self.h, m, C.byref(cnt), _dp(out["bo_prime"]), _dp(out["bo"]),
                                                    _dp(out["bo_pi"]), _dp(out["bo_pp"])))
        return out

    def qeq(self):
        q = np.empty(self.n)
        its = np.empty(self.nrep, np.int32)
        itt = np.empty(self.nrep, np.int32)
        rc = self._check(self.lib.reaxff_qeq(self.h, _dp(q), its.ctypes.data_as(C.POINTER(C.c_int32)),
                                             itt.ctypes.data_as(C.POINTER(C.c_int32))), allow=(E_NOT_CONVERGED,))
        return q, its, itt, rc == OK

    def forces(self, q=None):
        F = np.empty((self.n, 3))
        E = np.empty((self.nrep, NTERMS))
        W = np.empty((self.nrep, 6))
        if q is None:
            self._check(self.lib.reaxff_forces(self.h, _dp(F), _dp(E), _dp(W)), allow=(E_NOT_CONVERGED,))
        else:
            qq = np.ascontiguousarray(q, np.float64)
            self._check(self.lib.reaxff_forces_fixed_q(self.h, _dp(qq), _dp(F), _dp(E), _dp(W)))
        return F, E, W

    def step(self, nsteps, dt_fs=0.1, energies=True):
        et = np.empty((max(nsteps, 1), self.nrep)) if energies else None
        self._check(self.lib.reaxff_step(self.h, int(nsteps), float(dt_fs), _dp(et)))
        return et[:nsteps] if energies else None

    def step_dev(self, nsteps, dt_fs, etot_dev_ptr, stream_ptr):
        self._check(self.lib.reaxff_step_dev(self.h, int(nsteps), float(dt_fs), C.c_void_p(etot_dev_ptr),
                                             C.c_void_p(stream_ptr)))

    def last_launch_count(self):
        return int(self.lib.reaxff_last_launch_count(self.h))

    def reset_qeq_history(self):
        self.lib.reaxff_reset_qeq_history(self.h)

    def set_wait_limit(self, cycles):
        """Grid-barrier wait limit of the QEq kernel in SM cycles (<= 0: the default)."""
        self._check(self.lib.reaxff_set_wait_limit(self.h, int(cycles)))

    # ---- learned QEq warm start (marshalling only)
    MLP_NF, MLP_NPAR = 192, 16577

    def mlp_init(self, seed):
        self._check(self.lib.reaxff_mlp_init(self.h, int(seed)))

    def mlp_set_params(self, theta, mean, inv_std):
        th = np.ascontiguousarray(theta, np.float32).reshape(-1)
        mu = np.ascontiguousarray(mean, np.float32).reshape(-1)
        iv = np.ascontiguousarray(inv_std, np.float32).reshape(-1)
        if th.size != 4 * self.MLP_NPAR or mu.size != self.MLP_NF or iv.size != self.MLP_NF:
            raise ValueError("mlp_set_params: theta (4, 16577), mean (192,), inv_std (192,)")
        self._check(self.lib.reaxff_mlp_set_params(self.h, _fp(th), _fp(mu), _fp(iv)))

    def mlp_get_params(self):
        th = np.empty((4, self.MLP_NPAR), np.float32)
        mu = np.empty(self.MLP_NF, np.float32)
        iv = np.empty(self.MLP_NF, np.float32)
        self._check(self.lib.reaxff_mlp_get_params(self.h, _fp(th), _fp(mu), _fp(iv)))
        return th, mu, iv

    def mlp_descriptors(self):
        D = np.empty((self.n, self.MLP_NF), np.float32)
        self._check(self.lib.reaxff_mlp_descriptors(self.h, _fp(D)))
        return D

    def mlp_infer(self, D, types):
        D = np.ascontiguousarray(D, np.float32)
        t = np.ascontiguousarray(types, np.int32)
        y = np.empty(len(t), np.float32)
        self._check(self.lib.reaxff_mlp_infer(self.h, _fp(D), t.ctypes.data_as(C.POINTER(C.c_int32)), len(t), _fp(y)))
        return y

    def mlp_loss_grad(self, D, types, q):
        D = np.ascontiguousarray(D, np.float32)
        t = np.ascontiguousarray(types, np.int32)
        qq = np.ascontiguousarray(q, np.float32)
        g = np.empty((4, self.MLP_NPAR), np.float32)
        loss = C.c_double()
        self._check(self.lib.reaxff_mlp_loss_grad(self.h, _fp(D), t.ctypes.data_as(C.POINTER(C.c_int32)), _fp(qq),
                                                  len(t), _fp(g), C.byref(loss)))
        return loss.value, g

    def mlp_adam_step(self, grad, lr):
        g = np.ascontiguousarray(grad, np.float32).reshape(-1)
        self._check(self.lib.reaxff_mlp_adam_step(self.h, _fp(g), float(lr)))

    def mlp_reserve(self, nsnap):
        self._check(self.lib.reaxff_mlp_reserve(self.h, int(nsnap)))

    def mlp_collect(self):
        self._check(self.lib.reaxff_mlp_collect(self.h))

    def mlp_train(self, epochs, lr):
        loss = C.c_double()
        self._check(self.lib.reaxff_mlp_train(self.h, int(epochs), float(lr), C.byref(loss)))
        return loss.value

    def mlp_predict(self):
        q = np.empty(self.n)
        self._check(self.lib.reaxff_mlp_predict(self.h, _dp(q)))
        return q

    def species(self, bo_threshold=None, cap=4096):
        """Molecular species at the current positions: (mol_id int32[n], {(replica,
        counts of types 0..7): molecules})."""
        thr = None
        if bo_threshold is not None:
            thr = np.ascontiguousarray(bo_threshold, np.float64).reshape(MAXT * MAXT)
        mol = np.empty(self.n, np.int32)
        nmol = C.c_int64()
        rows = np.empty((cap, MAXT + 2), np.int32)
        ns = C.c_int32()
        self._check(self.lib.reaxff_species(self.h, None if thr is None else _dp(thr),
                                            mol.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(nmol), cap,
                                            rows.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(ns)))
        return mol, {tuple(int(v) for v in r[:-1]): int(r[-1]) for r in rows[:ns.value]}

    def bo_average_reset(self):
        self._check(self.lib.reaxff_bo_average_reset(self.h))

    def bo_average_sample(self):
        self._check(self.lib.reaxff_bo_average_sample(self.h))

    def bo_average_samples(self):
        return int(self.lib.reaxff_bo_average_samples(self.h))

    def get_bo_average(self):
        """Directed pairs seen since the last reset and their averaged bond orders:
        (i int32[m], j int32[m], shift int8[m, 3], avg float64[m])."""
        cnt = C.c_int64()
        self._check(self.lib.reaxff_get_bo_average(self.h, 0, C.byref(cnt), None, None, None, None))
        m = cnt.value
        i = np.empty(m, np.int32)
        j = np.empty(m, np.int32)
        s = np.empty((m, 3), np.int8)
        a = np.empty(m)
        self._check(self.lib.reaxff_get_bo_average(self.h, m, C.byref(cnt), i.ctypes.data_as(C.POINTER(C.c_int32)),
                                                   j.ctypes.data_as(C.POINTER(C.c_int32)),
                                                   s.ctypes.data_as(C.POINTER(C.c_int8)), _dp(a)))
        return i, j, s, a

    def species_average(self, bo_threshold=None, cap=4096):
        """species() on the time-averaged bond orders."""
        thr = None
        if bo_threshold is not None:
            thr = np.ascontiguousarray(bo_threshold, np.float64).reshape(MAXT * MAXT)
        mol = np.empty(self.n, np.int32)
        nmol = C.c_int64()
        rows = np.empty((cap, MAXT + 2), np.int32)
        ns = C.c_int32()
        self._check(self.lib.reaxff_species_average(self.h, None if thr is None else _dp(thr),
                                                    mol.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(nmol), cap,
                                                    rows.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(ns)))
        return mol, {tuple(int(v) for v in r[:-1]): int(r[-1]) for r in rows[:ns.value]}

    def autotune(self, cache_path=None):
        """Pick launch schedules by timing; returns (torsion lanes, nonbonded, filter,
        bond list, angles, H-bonds, angle lanes, QEq beside the charge-free terms)."""
        sch = np.empty(8, np.int32)
        self._check(self.lib.reaxff_autotune(self.h, None if cache_path is None else str(cache_path).encode(),
                                             sch.ctypes.data_as(C.POINTER(C.c_int32))))
        return tuple(int(v) for v in sch)

    def qeq_warm_choice(self):
        """Per replica: 1 where the last QEq solve kept the learned guess for s."""
        u = np.empty(self.nrep, np.int32)
        self._check(self.lib.reaxff_qeq_warm_choice(self.h, u.ctypes.data_as(C.POINTER(C.c_int32))))
        return u

    def qeq_spmv_total(self):
        """SpMVs (one read of H for both systems) of all QEq solves so far."""
        v = self.lib.reaxff_qeq_spmv_total(self.h)
        if v < 0:
            raise ReaxFFError(E_CUDA, "reaxff_qeq_spmv_total failed")
        return int(v)

    def last_qeq_iters(self):
        its = np.empty(self.nrep, np.int32)
        itt = np.empty(self.nrep, np.int32)
        self._check(self.lib.reaxff_last_qeq_iters(self.h, its.ctypes.data_as(C.POINTER(C.c_int32)),
                                                   itt.ctypes.data_as(C.POINTER(C.c_int32))))
        return its, itt

    def profile_enable(self, on=True):
        """True / 1: stage timers with the stages in order; 2: the overlapped order with its
        two path spans; False / 0: off."""
        self.lib.reaxff_profile_enable(self.h, int(on))

    def profile_read(self):
        """{stage name: (accumulated ms, timed launches)} from the CUDA-event stage timers."""
        ms = np.zeros(32)
        calls = np.zeros(32, np.int64)
        k = self.lib.reaxff_profile_read(self.h, 32, _dp(ms), calls.ctypes.data_as(C.POINTER(C.c_int64)))
        return {self.lib.reaxff_stage_name(i).decode(): (float(ms[i]), int(calls[i])) for i in range(k)}


def virial_matrix(w6):
    """(xx, yy, zz, xy, xz, yz) -> symmetric 3x3."""
    xx, yy, zz, xy, xz, yz = w6
    return np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]])
