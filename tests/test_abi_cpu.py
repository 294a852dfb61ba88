"""C-ABI library checks that need no GPU: it builds, loads, exports every declared
symbol, and its struct layouts match the Python binding (CPU only)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in ("reaxff.h",)]


@pytest.fixture(scope="module")
def lib():
    from paper_1706_07772_gb300 import build as B
    B.build()
    import paper_1706_07772_gb300.reaxff as rx
    return rx.load()


def _declared():
    names = set()
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(reaxff_\w+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_struct_layouts_match(lib):
    import ctypes as C

    import paper_1706_07772_gb300.reaxff as rx
    assert lib.reaxff_sizeof_params() == C.sizeof(rx.Params)
    assert lib.reaxff_sizeof_options() == C.sizeof(rx.Options)
    for name, _ in rx.Params._fields_:
        assert lib.reaxff_params_offset(name.encode()) == getattr(rx.Params, name).offset
    assert lib.reaxff_params_offset(b"no_such_field") == -1


def test_params_packing_roundtrip(params):
    import paper_1706_07772_gb300.reaxff as rx
    P = rx.make_params(params)
    assert P.ntypes == 4
    assert P.th00[1][0][2] == params["th00"][1, 0, 2]
    assert P.k_e == params["k_e"]
    assert list(P.hb)[:4] == [0, 1, 2, 2]


def test_term_mask_bits():
    import paper_1706_07772_gb300.reaxff as rx
    assert rx.term_mask("bond") == 1
    assert rx.term_mask("pol") == 1 << 12
    assert rx.term_mask(*rx.TERMS) == (1 << 13) - 1


def test_no_cpu_fallback_when_library_missing(tmp_path):
    import paper_1706_07772_gb300.reaxff as rx
    with pytest.raises(ImportError):
        rx._lib = None
        rx.load(str(tmp_path / "missing.so"))
    rx._lib = None
    rx.load()


def test_virial_matrix_symmetric():
    import paper_1706_07772_gb300.reaxff as rx
    W = rx.virial_matrix(np.arange(6.0))
    assert np.array_equal(W, W.T)
    assert W[0, 1] == 3 and W[0, 2] == 4 and W[1, 2] == 5
