"""The allocation-free far-list builder (reaxff_far_list_noalloc) against the context
path (reaxff_build_lists + reaxff_get_lists).

Callers that cannot allocate device memory at run time (their own memory pool owns the
GPU, or a cudaMalloc's device-wide synchronisation would stall other work) use the
allocation-free entry point; its lists must be the ones the regular path builds. Two
calls in a row on different systems check that the shared scratch array's leftovers
from one call do not leak into the next.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _lib():
    from paper_1706_07772_gb300 import build as B
    B.build()
    import paper_1706_07772_gb300.reaxff as rx
    lib = rx.load()
    f = lib.reaxff_far_list_noalloc
    f.restype = C.c_int
    vp = C.c_void_p
    f.argtypes = [C.POINTER(rx.Params), C.POINTER(rx.Options), vp, vp, vp, vp, C.c_int64,
                  C.POINTER(C.c_double), C.c_int32, vp, vp, vp, vp, vp, C.POINTER(C.c_char_p)]
    return rx, f


def _keys(i, j, s, n):
    return np.sort(oracle.sort_key(np.asarray(i, np.int64), np.asarray(j, np.int64), np.asarray(s, np.int64), n))


def test_noalloc_far_list_matches_context_two_calls():
    torch = pytest.importorskip("torch")
    rx, f = _lib()
    P = synth.make_params()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    for name in ("petn464", "cluster300"):
        w = synth.workload(name)
        n = len(w["types"])
        ctx = rx.ReaxFF(P, w["types"], w["box"], w["options"], precision=rx.FP64)
        ctx.set_state(w["x"])
        ctx.build_lists()
        want = _keys(*ctx.get_lists(rx.LIST_FAR), n)
        x, _, _ = ctx.get_state()          # the context's wrapped positions
        ctx.close()
        X = torch.tensor(np.ascontiguousarray(x[:, 0]), dtype=torch.float64, device=dev)
        Y = torch.tensor(np.ascontiguousarray(x[:, 1]), dtype=torch.float64, device=dev)
        Z = torch.tensor(np.ascontiguousarray(x[:, 2]), dtype=torch.float64, device=dev)
        T = torch.tensor(w["types"], dtype=torch.int32, device=dev)
        cap = 640
        cnt = torch.full((n,), -1, dtype=torch.int32, device=dev)
        J = torch.full((n * cap,), -1, dtype=torch.int32, device=dev)
        S = torch.zeros(n * cap, dtype=torch.uint8, device=dev)
        H = torch.zeros(n * cap, dtype=torch.float64, device=dev)
        box = (C.c_double * 3)(*w["box"])
        msg = C.c_char_p()
        Pc, Oc = rx.make_params(P), rx.make_options(w["options"])
        rc = f(C.byref(Pc), C.byref(Oc), T.data_ptr(), X.data_ptr(), Y.data_ptr(), Z.data_ptr(), n, box, cap,
               cnt.data_ptr(), J.data_ptr(), S.data_ptr(), H.data_ptr(), stream.cuda_stream, C.byref(msg))
        assert rc == 0, msg.value
        cnt_h = cnt.cpu().numpy()
        J_h = J.cpu().numpy().reshape(n, cap)
        S_h = S.cpu().numpy().reshape(n, cap).astype(np.int64)
        H_h = H.cpu().numpy().reshape(n, cap)
        ii = np.concatenate([np.full(c, i) for i, c in enumerate(cnt_h)])
        jj = np.concatenate([J_h[i, :c] for i, c in enumerate(cnt_h)])
        cc = np.concatenate([S_h[i, :c] for i, c in enumerate(cnt_h)])
        ss = np.stack([cc // 9 - 1, (cc // 3) % 3 - 1, cc % 3 - 1], 1)
        assert np.array_equal(_keys(ii, jj, ss, n), want)
        # H entry of every (i, j, s) against the oracle's matrix entry at the same positions
        hv = np.concatenate([H_h[i, :c] for i, c in enumerate(cnt_h)])
        m = oracle.Model(P, w["types"], w["box"], w["options"])
        href = m.qeq_entries(x, ii, jj, ss)
        assert np.abs(hv - href).max() <= 1e-12 * np.abs(href).max()


def test_noalloc_rejects_sizes_beyond_the_limit():
    torch = pytest.importorskip("torch")
    rx, f = _lib()
    P = synth.make_params()
    w = synth.workload("petn464")
    dev = torch.device("cuda", 0)
    buf = torch.zeros(16, dtype=torch.float64, device=dev)
    box = (C.c_double * 3)(*w["box"])
    msg = C.c_char_p()
    Pc, Oc = rx.make_params(P), rx.make_options(w["options"])
    p = buf.data_ptr()
    rc = f(C.byref(Pc), C.byref(Oc), p, p, p, p, 65537, box, 8, p, p, p, p, None, C.byref(msg))
    assert rc == rx.E_INVALID and b"65536" in msg.value


def test_noalloc_rejects_invalid_device_inputs():
    """A type outside [0, ntypes), or a position outside [0, L), is found by the entry
    point's device-side check before any list kernel runs: E_INVALID, and a valid call
    afterwards still succeeds."""
    torch = pytest.importorskip("torch")
    rx, f = _lib()
    P = synth.make_params()
    w = synth.workload("petn464")
    n = len(w["types"])
    dev = torch.device("cuda", 0)
    x = np.mod(w["x"], w["box"])
    x = np.where(x >= w["box"], x - w["box"], x)
    box = (C.c_double * 3)(*w["box"])
    Pc, Oc = rx.make_params(P), rx.make_options(w["options"])
    cap = 640
    cnt = torch.zeros(n, dtype=torch.int32, device=dev)
    J = torch.zeros(n * cap, dtype=torch.int32, device=dev)
    S = torch.zeros(n * cap, dtype=torch.uint8, device=dev)
    H = torch.zeros(n * cap, dtype=torch.float64, device=dev)

    def call(types, pos):
        T = torch.tensor(types, dtype=torch.int32, device=dev)
        X, Y, Z = (torch.tensor(np.ascontiguousarray(pos[:, k]), dtype=torch.float64, device=dev) for k in range(3))
        msg = C.c_char_p()
        rc = f(C.byref(Pc), C.byref(Oc), T.data_ptr(), X.data_ptr(), Y.data_ptr(), Z.data_ptr(), n, box, cap,
               cnt.data_ptr(), J.data_ptr(), S.data_ptr(), H.data_ptr(), None, C.byref(msg))
        torch.cuda.synchronize()
        return rc, msg.value

    bad_t = w["types"].copy()
    bad_t[17] = 4
    rc, msg = call(bad_t, x)
    assert rc == rx.E_INVALID and b"type" in msg
    bad_t[17] = -1
    rc, msg = call(bad_t, x)
    assert rc == rx.E_INVALID and b"type" in msg
    bad_x = x.copy()
    bad_x[3, 1] = w["box"][1] + 0.5                       # not wrapped into the box
    rc, msg = call(w["types"], bad_x)
    assert rc == rx.E_INVALID and b"position" in msg
    bad_x[3, 1] = -0.25
    rc, msg = call(w["types"], bad_x)
    assert rc == rx.E_INVALID and b"position" in msg
    rc, msg = call(w["types"], x)
    assert rc == 0, msg
    # n * cap beyond 32-bit row offsets is refused on the host
    p = H.data_ptr()
    msg = C.c_char_p()
    rc = f(C.byref(Pc), C.byref(Oc), p, p, p, p, 65536, box, 40000, p, p, p, p, None, C.byref(msg))
    assert rc == rx.E_INVALID and b"cap" in msg.value
