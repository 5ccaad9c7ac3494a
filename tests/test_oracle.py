"""The FP64 oracle against its pins (no GPU), and a mutation test showing that a
plausible mistake planted anywhere in the oracle fails at least one pin."""
import os

import pytest

import oracle
import oracle_pins as pins
from oracle import build as obuild

CHECKS = sorted(n for n in dir(pins) if n.startswith("check_"))


@pytest.mark.parametrize("name", CHECKS)
def test_pin(name):
    getattr(pins, name)()


# (description, text in hamr_oracle.c, replacement)
MUTANTS = [
    ("precession sign", "double pref = -p->gamma", "double pref = p->gamma"),
    ("missing 1/(1+alpha^2)", "/ (1.0 + p->alpha * p->alpha)", "/ 1.0"),
    ("dropped damping term", "pref * (sxb[d] + p->alpha * sxsxb[d])", "pref * sxb[d]"),
    ("anisotropy factor 2", "double ani = 2.0 * p->ku", "double ani = 1.0 * p->ku"),
    ("anisotropy on x", "B[0] = ex[0] / p->mu_s + Bapp[0];", "B[0] = ex[0] / p->mu_s + Bapp[0] + ani;"),
    ("thermal variance factor 2", "sqrt(2.0 * p->alpha * ORC_KB", "sqrt(p->alpha * ORC_KB"),
    ("Euler corrector", "S[3 * i + d] + 0.5 * p->dt * (f1[3 * i + d] + f2[d])", "S[3 * i + d] + p->dt * f2[d]"),
    ("no renormalisation", "        normalise(S + 3 * i);\n    }\n    free(Bth)", "    }\n    free(Bth)"),
    ("one J for all shells", "double Jk = p->J[shells[k]];", "double Jk = p->J[0];"),
    ("exchange uses S_i", "const double *Sj = S + 3 * js[k];", "const double *Sj = S + 3 * i;"),
    ("Box-Muller sin->cos", "r1 * sin(2.0 * ORC_PI * u[1])", "r1 * cos(2.0 * ORC_PI * u[1])"),
    ("Philox multiplier", "0xCD9E8D57u * (uint64_t)c2", "0xCD9E8D55u * (uint64_t)c2"),
    ("laser FWHM law", "-4.0 * log(2.0) * r2", "-log(2.0) * r2"),
    ("field ramp direction", "return prev + (cur - prev) * w;", "return cur + (prev - cur) * w;"),
    ("shell tolerance", "<= 1e-6 * p->shell_dist[s]", "<= 1e-1 * p->shell_dist[s]"),
    ("grain coupling", "if (grain[j] != grain[i]) continue;", ""),
    ("predictor noise scale", "for (int d = 0; d < 3; ++d) B[d] += Bth[3 * i + d];\n        orc_llg_rhs(p, S + 3 * i",
     "for (int d = 0; d < 3; ++d) B[d] += 2.0 * Bth[3 * i + d];\n        orc_llg_rhs(p, S + 3 * i"),
    ("magnetisation counts voids", "if (c->grain[i] < 0) continue;\n        for (int d = 0; d < 3; ++d) m[d]",
     "for (int d = 0; d < 3; ++d) m[d]"),
    ("energy counts each bond twice", "E -= 0.5 * p->J[c->shell[k]]", "E -= p->J[c->shell[k]]"),
    ("grain sums drop the last grain", "if (g < 0 || g >= n_grains) continue;",
     "if (g < 0 || g >= n_grains - 1) continue;"),
]


@pytest.mark.parametrize("desc,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(desc, old, new, tmp_path, monkeypatch):
    src = open(obuild.SRC).read()
    assert src.count(old) == 1, desc
    mut = tmp_path / "mutant.c"
    mut.write_text(src.replace(old, new))
    lib = obuild.build(src=str(mut), lib=str(tmp_path / "libmutant.so"), force=True)
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
