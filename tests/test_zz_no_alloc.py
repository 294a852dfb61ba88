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
        hv = np.concatenate([H_h[i, :c] for i, c in enumerate(cnt_h)])
        assert np.all(np.isfinite(hv)) and np.all(hv > -1e-12)


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
