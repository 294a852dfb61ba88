"""Strength of the oracle's term pins (CPU only): each plausible mistake below is planted in a
copy of the oracle's energy (a sign, an index, a dropped or changed factor) and at least one
pin of tests/test_oracle_term_pins.py must then fail. The mistakes are planted in the oracle
on the CPU; nothing here touches the GPU path."""
import importlib.util
import os
import types

import pytest

import oracle
from oracle import reaxff_oracle as ro

HERE = os.path.dirname(os.path.abspath(__file__))

MUTATIONS = [
 ("f2 sign", "f2 = torch.exp(-pb1 * dpi) + torch.exp(-pb1 * dpj)", "f2 = torch.exp(pb1 * dpi) + torch.exp(pb1 * dpj)"),
 ("f3 sign", "f3 = -(1.0 / pb2)", "f3 = (1.0 / pb2)"),
 ("f1 index", "(vj + f2) / (vj + f2 + f3)", "(vi + f2) / (vi + f2 + f3)"),
 ("f4 p5 sign", "f4 = _sig(-p3 * (p4 * bop * bop - dpboc[bi]) + p5)", "f4 = _sig(-p3 * (p4 * bop * bop - dpboc[bi]) - p5)"),
 ("f5 index", "dpboc[bj]) + p5)", "dpboc[bi]) + p5)"),
 ("BOpi f1 power", "BOpi = bp * f1 * f1 * f4 * f5", "BOpi = bp * f1 * f4 * f5"),
 ("BOpp f1 power", "BOpp = bpp * f1 * f1 * f4 * f5", "BOpp = bpp * f1 * f4 * f5"),
 ("Ebond sign", "pbe1 * (1.0 - torch.pow(bsafe, pbe2))", "pbe1 * (torch.pow(bsafe, pbe2) - 1.0)"),
 ("Ebond pi", "- _t(P[\"De_p\"][ti, tj]) * BOpi", "- _t(P[\"De_p\"][ti, tj]) * BOs"),
 ("nlp T", "el = 2.0 + Dele - 2.0 * Tr", "el = 2.0 + Dele + 2.0 * Tr"),
 ("nlp opt", "nlp_opt = 0.5 * (_t(P[\"vale\"][ty]) - val)", "nlp_opt = 0.5 * (_t(P[\"vale\"][ty]) + val)"),
 ("Elp switch", "torch.sigmoid(75.0 * Dlp)", "torch.sigmoid(-75.0 * Dlp)"),
 ("S index", "S = S.index_add(0, torch.as_tensor(bi), dd[bj] * (BOpi + BOpp))", "S = S.index_add(0, torch.as_tensor(bi), dd[bi] * (BOpi + BOpp))"),
 ("dlpc exp sign", "torch.exp(P[\"p_ovun4\"] * S))", "torch.exp(-P[\"p_ovun4\"] * S))"),
 ("Eover sig", "_sig(pov2 * Dlpc)", "_sig(-pov2 * Dlpc)"),
 ("Eover val", "Dlpc / (Dlpc + val + 1e-8)", "Dlpc / (Dlpc + 1.0 + 1e-8)"),
 ("Eunder p6", "(1.0 - torch.exp(P[\"p_ovun6\"] * Dlpc))", "(1.0 - torch.exp(-P[\"p_ovun6\"] * Dlpc))"),
 ("Eunder S", "(1.0 + P[\"p_ovun7\"] * torch.exp(P[\"p_ovun8\"] * S))", "(1.0 + P[\"p_ovun7\"] * torch.exp(-P[\"p_ovun8\"] * S))"),
 ("SBO nlp sign", "(-Dang - P[\"p_val8\"] * nlp)", "(-Dang + P[\"p_val8\"] * nlp)"),
 ("SBO pi", "pisum = atom_sum(BOpi + BOpp)", "pisum = atom_sum(BOpi)"),
 ("SBO2 branch", "s_hi = torch.clamp(2.0 - SBO, 1e-30, 1.0)", "s_hi = torch.clamp(SBO - 1.0, 1e-30, 1.0)"),
 ("theta0", "(1.0 - torch.exp(-P[\"p_val10\"] * (2.0 - SBO2[jj])))", "(1.0 - torch.exp(-P[\"p_val10\"] * (SBO2[jj])))"),
 ("f7 power", "f7a = 1.0 - torch.exp(-pv3 * torch.pow(BOa, pv4))", "f7a = 1.0 - torch.exp(-pv3 * BOa)"),
 ("f8 p7 sign", "torch.exp(-_t(P[\"p_val7\"][ti_, tj_, tk_]) * Dj)", "torch.exp(_t(P[\"p_val7\"][ti_, tj_, tk_]) * Dj)"),
 ("f9 p4 sign", "torch.exp(P[\"p_pen4\"] * Dd)", "torch.exp(-P[\"p_pen4\"] * Dd)"),
 ("pen 2", "torch.exp(-P[\"p_pen2\"] * (BOa - 2.0) ** 2)", "torch.exp(-P[\"p_pen2\"] * (BOa - 1.0) ** 2)"),
 ("coa index", "(sumBO[kk] - BOb)", "(sumBO[jj] - BOb)"),
 ("coa sig", "_sig(P[\"p_coa2\"] * Dj)", "_sig(-P[\"p_coa2\"] * Dj)"),
 ("coa 1.5", "torch.exp(-P[\"p_coa4\"] * (BOb - 1.5) ** 2)", "torch.exp(-P[\"p_coa4\"] * (BOb - 1.0) ** 2)"),
 ("f10 index", "(1.0 - torch.exp(-pt2 * BO2))", "(1.0 - torch.exp(-pt2 * BO1))"),
 ("f11 sign", "torch.exp(P[\"p_tor4\"] * Dsum)", "torch.exp(-P[\"p_tor4\"] * Dsum)"),
 ("V2 form", "(2.0 - BOpi[bc] - f11)", "(BOpi[bc] - 1.0 + f11)"),
 ("V2 cos", "* (1.0 - c2w)", "* (1.0 + c2w)"),
 ("conj 1.5", "torch.exp(-pc2 * (BO2 - 1.5) ** 2)", "torch.exp(-pc2 * (BO2 - 1.0) ** 2)"),
 ("Dang val", "Dang = sumBO - _t(P[\"valang\"][ty])", "Dang = sumBO - _t(P[\"val\"][ty])"),
]


def _pins():
    spec = importlib.util.spec_from_file_location("term_pins_for_mutants", os.path.join(HERE, "test_oracle_term_pins.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    calls = []
    for name, fn in vars(mod).items():
        if not (name.startswith("test_") and callable(fn)):
            continue
        combos = [{}]
        for m in getattr(fn, "pytestmark", []):
            if m.name != "parametrize":
                continue
            names = [a.strip() for a in m.args[0].split(",")]
            combos = [dict(c, **dict(zip(names, v if len(names) > 1 else (v,)))) for c in combos for v in m.args[1]]
        calls += [(fn, c) for c in combos]
    return calls


@pytest.fixture(scope="module")
def pins():
    return _pins()


@pytest.fixture(scope="module")
def source():
    with open(ro.__file__) as f:
        return f.read()


def test_pins_pass_on_the_oracle_as_written(params, pins):
    for fn, kw in pins:
        fn(params, **kw)


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(params, pins, source, monkeypatch, name, old, new):
    assert source.count(old) == 1, name
    mutant = types.ModuleType("oracle_mutant")
    exec(compile(source.replace(old, new), ro.__file__ + " (mutant)", "exec"), mutant.__dict__)
    monkeypatch.setattr(oracle, "Model", mutant.Model)
    for fn, kw in pins:
        try:
            fn(params, **kw)
        except Exception:            # an assertion, or the mutant's arithmetic breaking down
            return
    pytest.fail("no pin failed with the planted mistake: " + name)
