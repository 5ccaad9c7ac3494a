"""The multiscale-window oracle against its pins (no GPU), and a mutation test: a plausible
mistake planted anywhere in oracle/hamr_ms_oracle.c fails at least one pin."""
import pytest

import ms_pins as pins
import oracle
from oracle import build as obuild

CHECKS = [c.__name__ for c in pins.FAST_CHECKS]


@pytest.mark.parametrize("name", CHECKS)
def test_ms_pin(name):
    getattr(pins, name)()


# (description, text in hamr_ms_oracle.c, replacement)
MUTANTS = [
    ("atomistic side drops the interface bond", "v = c->m + 3 * q;\n", "v = c->m + 3 * q;\n            continue;\n"),
    ("micromagnetic side ignores window cells", "if (c->grain[qn] != c->grain[q]) continue;",
     "if (c->grain[qn] != c->grain[q] || (x >= c->ox && x < c->ox + p->wx)) continue;"),
    ("damping law without the 1/3", "return p->lambda * (1.0 - Tc / (3.0 * p->T_C));",
     "return p->lambda * (1.0 - Tc / p->T_C);"),
    ("A(T) with m_e instead of m_e^2", "double cex = 2.0 * p->A0 * me * me / (p->Ms0 * me)",
     "double cex = 2.0 * p->A0 * me / (p->Ms0 * me)"),
    ("K(T) with m_e^2 instead of m_e^3", "cK = 2.0 * p->K0 * me * me * me / (p->Ms0 * me)",
     "cK = 2.0 * p->K0 * me * me / (p->Ms0 * me)"),
    ("RK4 weights", "wstage[4] = {1.0, 2.0, 2.0, 1.0}", "wstage[4] = {1.0, 1.0, 1.0, 1.0}"),
    ("RK4 stage points", "cstage[4] = {0.5, 0.5, 1.0, 0.0}", "cstage[4] = {1.0, 1.0, 1.0, 0.0}"),
    ("cone law constant", "(5.0 * ORC_PI / 9.0)", "(4.0 * ORC_PI / 9.0)"),
    ("cone uniform in cos(theta)", "double th = u0 * theta_max", "double th = acos(1.0 - u0 * (1.0 - cos(theta_max)))"),
    ("m_e without the field", "b = mu_s * B / (ORC_KB * T)", "b = 0.0 * B / (ORC_KB * T)"),
    ("m_e mean-field factor 3", "double a = 3.0 * T_C / T", "double a = T_C / T"),
    ("Eq. 6 not normalised", "c->m[3 * q + d] = n > 0.0 ? s[d] / n : 0.0;", "c->m[3 * q + d] = s[d];"),
    ("shift keeps the old sites", "c->S[3 * (i + r + nxw * (j + nyw * k)) + d]", "c->S[3 * (i + nxw * (j + nyw * k)) + d]"),
    ("thermalised column at the trailing end", "thermalise(c, c->ox + c->p.wx - 1, c->ox + c->p.wx, t,",
     "thermalise(c, c->ox, c->ox + 1, t,"),
    ("window thermal variance uses alpha(T)", "double sigma = sqrt(2.0 * p->lambda * ORC_KB * T",
     "double sigma = sqrt(2.0 * orc_ms_alpha(p, T) * ORC_KB * T"),
    ("window anisotropy factor", "B[2] = ex[2] / p->mu_s + 2.0 * p->ku / p->mu_s * Si[2]",
     "B[2] = ex[2] / p->mu_s + p->ku / p->mu_s * Si[2]"),
    ("window target off by half a window", "floor(xc / p->cell - 0.5 * p->wx + 0.5)", "floor(xc / p->cell + 0.5)"),
    ("read-back counts non-magnetic cells", "if (c->grain[q] < 0) continue;\n                    sum +=",
     "sum +="),
    ("read-back bit sign", "bits[b] = signal[b] < 0.0 ? 1 : 0;", "bits[b] = signal[b] > 0.0 ? 1 : 0;"),
    ("head profile upside down", "double Pz = 0.5 * (1.0 - tanh(", "double Pz = 0.5 * (1.0 + tanh("),
    ("in-plane component without polarity", "B[0] += p->prof_Bx0 * s * Px;", "B[0] += p->prof_Bx0 * Px;"),
    ("window ignores the head profile",
     "orc_ms_field(p, ((double)c->ox * r + i + 0.5) * a, t, Bapp);\n        site_exchange(c, c->S,",
     "orc_applied_field(&p->drv, t, Bapp);\n        site_exchange(c, c->S,"),
    ("cells ignore the head profile", "orc_ms_field(p, (q % p->ncx + 0.5) * p->cell, t, Bq + 3 * q);",
     "orc_applied_field(&p->drv, t, Bq + 3 * q);"),
    ("Newell f term sign", "r -= x * y * z * atan_ratio(y * z, x * R);", "r += x * y * z * atan_ratio(y * z, x * R);"),
    ("Newell g last term", "r -= x * y * R / 3.0;", "r -= x * y * R / 6.0;"),
    ("second-difference weights", "static const double c[3] = {-1.0, 2.0, -1.0};",
     "static const double c[3] = {1.0, -2.0, 1.0};"),
    ("far-field dipole sign", "pre = -V / (4.0 * ORC_PI * r * r * r)", "pre = V / (4.0 * ORC_PI * r * r * r)"),
    ("window cells enter as directions", "M[3 * q + d] += p->mu_s / V * Si[d];", "M[3 * q + d] += Si[d];"),
    ("window misses the demagnetising field",
     "B[2] = ex[2] / p->mu_s + 2.0 * p->ku / p->mu_s * Si[2] + Bapp[2] + Bth[3 * s + 2] + bd[2];",
     "B[2] = ex[2] / p->mu_s + 2.0 * p->ku / p->mu_s * Si[2] + Bapp[2] + Bth[3 * s + 2];"),
    ("cells miss the demagnetising field", "double B[3] = {cex * lap[0] + Bapp[0] + bd[0],",
     "double B[3] = {cex * lap[0] + Bapp[0],"),
    ("re-placed window keeps its cells", "    if (c->live) average_cells(c, c->ox, c->ox + c->p.wx);\n", ""),
    ("new drivers ignored", "    c->p = *p;\n    c->p.drv.bits = bits;", "    c->p.drv.bits = bits;"),
    ("new drivers reset the step count", "    c->p = *p;\n    c->p.drv.bits = bits;",
     "    c->p = *p;\n    c->p.drv.bits = bits;\n    c->step = 0;"),
    ("simulated region one column longer", "cx < (int64_t)c->ox + c->p.wx + g", "cx <= (int64_t)c->ox + c->p.wx + g"),
    ("frozen cells evolved", "((q) % p->ncx < c->ox || (q) % p->ncx >= c->ox + p->wx) && in_region(c, (q) % p->ncx))",
     "((q) % p->ncx < c->ox || (q) % p->ncx >= c->ox + p->wx))"),
    ("frozen cells' m_e never stored", "    store_me(c, (double)c->step * c->p.drv.dt);\n", ""),
]


@pytest.mark.parametrize("desc,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_ms_mutant_is_caught(desc, old, new, tmp_path, monkeypatch):
    src = open(obuild.MS_SRC).read()
    assert src.count(old) == 1, desc
    mut = tmp_path / "ms_mutant.c"
    mut.write_text(src.replace(old, new))
    lib = obuild.build(lib=str(tmp_path / "libmutant.so"), force=True, ms_src=str(mut))
    monkeypatch.setattr(oracle, "_lib", None)
    monkeypatch.setattr(obuild, "build", lambda *a, **k: lib)
    caught = None
    for chk in pins.FAST_CHECKS:
        try:
            chk()
        except AssertionError:
            caught = chk.__name__
            break
    monkeypatch.setattr(oracle, "_lib", None)
    assert caught is not None, "mutant '%s' passed every pin" % desc
