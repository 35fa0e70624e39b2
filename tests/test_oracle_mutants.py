"""The oracle's magnitude pins catch the slips they are meant to catch.

Each case plants one plausible mistake in a copy of the oracle's C source
(on the CPU, in a temporary directory), builds it, and checks that the pin
of test_oracle_pins that guards that passage no longer holds:

  * Eq. eqn_ladd_lubrikation with 3 pi for 6 pi, with R^2 in place of
    R^4 / (2R)^2, or with the viscosity of the red component only;
  * Eq. masscorr with the fluid-node count in place of the number of all
    lattice sites N, or without the density ratio.
"""
import os
import subprocess

import numpy as np
import pytest

from oracle import build as obuild
from oracle import ref

from test_oracle_pins import lubrication_cases, masscorr_factors

SRC = os.path.join(os.path.dirname(obuild.__file__), "lbref.c")

LUB = "double mag = -6.0 * M_PI * nu * pow(R, 4) / (4.0 * R * R) * dot3(rh, du) * (1.0 / he - 1.0 / P->lub_cut);"
NU = "double nu = (1.0 / 3.0) * (0.5 * (P->tau[0] + P->tau[1]) - 0.5);"
MC = "corr[c] = 1.0 - s->p.mass_corr_c0 * (rsum / s->p.rho_init[c]) * (mass_now[c] - s->mass0[c]) / (double)N;"

MUTANTS = {
    "lub_3pi": (LUB, LUB.replace("-6.0 * M_PI", "-3.0 * M_PI")),
    "lub_R2": (LUB, LUB.replace("pow(R, 4) / (4.0 * R * R)", "R * R")),
    "lub_nu_red": (NU, NU.replace("0.5 * (P->tau[0] + P->tau[1])", "P->tau[0]")),
    "mc_nfluid": (MC, "{ int64_t nf_ = 0; for (int64_t k_ = 0; k_ < N; k_++) nf_ += s->owner[k_] == -1; "
                      + MC.replace("/ (double)N;", "/ (double)nf_;") + " }"),
    "mc_no_ratio": (MC, MC.replace(" * (rsum / s->p.rho_init[c])", "")),
}


def _lubrication_ok():
    return all(abs(got - want) < 1e-12 * want for got, want in lubrication_cases())


def _masscorr_ok():
    measured, expected = masscorr_factors()
    return all(np.allclose(measured[c], expected[c], rtol=0, atol=1e-13) for c in range(2))


@pytest.fixture
def mutant(tmp_path, monkeypatch):
    """Build the oracle with one planted slip and make ref use it."""

    def make(name):
        old, new = MUTANTS[name]
        src = open(SRC).read()
        assert src.count(old) == 1, "pattern of %s not found once in the oracle source" % name
        path = tmp_path / ("lbref_%s.c" % name)
        path.write_text(src.replace(old, new))
        lib = tmp_path / ("liblbref_%s.so" % name)
        subprocess.check_call(["gcc", "-std=gnu11", "-O1", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-I", os.path.dirname(SRC), "-o", str(lib), str(path), "-lm"])
        monkeypatch.setattr(ref, "_lib", None)
        monkeypatch.setattr(ref._build, "build", lambda force=False: str(lib))
        ref.lib()

    yield make
    monkeypatch.undo()
    ref._lib = None


def test_unmutated_oracle_passes_both_pins():
    assert _lubrication_ok()
    assert _masscorr_ok()


@pytest.mark.parametrize("name", ["lub_3pi", "lub_R2", "lub_nu_red"])
def test_lubrication_pin_catches(mutant, name):
    mutant(name)
    assert not _lubrication_ok()
    assert _masscorr_ok()


@pytest.mark.parametrize("name", ["mc_nfluid", "mc_no_ratio"])
def test_mass_correction_pin_catches(mutant, name):
    mutant(name)
    assert not _masscorr_ok()
    assert _lubrication_ok()
