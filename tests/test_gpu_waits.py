"""Bounded device-side waits (the E_TIMEOUT path of the C ABI): the persistent QEq kernel's
grid barrier gives up after a cycle limit, the call reports REAXFF_E_TIMEOUT and the
context stays usable. The wait runs out by a small limit set through the ABI; nothing
faults, traps or hangs the GPU."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_wait_limit_timeout_path(params):
    """The QEq kernel's grid-barrier waits are bounded: with a limit of 100 SM cycles a wait
    runs out, the call returns REAXFF_E_TIMEOUT (every block left the kernel through its
    bounded wait, so the call returned at all), and with the default limit restored the
    same context solves to the dense oracle solution again."""
    import paper_1706_07772_gb300.reaxff as rx
    w = synth.workload("petn464")
    o = dict(w["options"], qeq_tol=1e-10)
    m = oracle.Model(params, w["types"], w["box"], o)
    qd = m.qeq_dense(w["x"], m.lists(w["x"]))["q"]
    for prec in (rx.FP64, rx.MIXED):
        c = rx.ReaxFF(params, w["types"], w["box"], o, precision=prec)
        c.set_state(w["x"], w["v"])
        c.set_wait_limit(100)
        for _ in range(2):
            with pytest.raises(rx.ReaxFFError) as e:
                c.qeq()
            assert e.value.code == rx.E_TIMEOUT
        c.set_wait_limit(0)
        q, its, itt, conv = c.qeq()
        assert conv
        assert np.abs(q - qd).max() < (1e-8 if prec == rx.FP64 else 1e-5)
        c.close()
