"""Mass over long runs in each population storage, with no cover or
uncover events (fixed spheres), where the method conserves each
component's mass exactly and only rounding moves it.

FP64 storage keeps it to rounding of FP64 sums.  FP32 storage sums its
densities in FP32, and 16-bit deviation storage also rounds every stored
population; the rest population (the density minus the 18 stored values)
takes that rounding, so each step moves a node's mass by a few 2^-24 of
it.  On a generic state those errors do not add coherently: the drift
grows like a random walk.  The test allows ten times a random walk of
4 * 2^-24 per step, 10 sqrt(steps) * 4 * 2^-24 relative (2.4e-4 after
10^4 steps); measured on a GB300 after 10^4 steps: FP32 -2.1e-6,
FP16 7.4e-6, BF16 1.4e-5, FP64 2e-15.

Setup: 64^3 two-component mixture (0.35 / 0.35, node noise 0.05,
g = 0.08, so it demixes), 40 fixed spheres of radius 5."""
import math

import numpy as np
import pytest

import lbinputs

pytestmark = pytest.mark.gpu

SHAPE = (64, 64, 64)
CHECKS = (1000, 3000, 10000)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16", "bf16"])
def test_mass_drift_is_rounding_only(precision):
    from paper_1004_4414_gb300 import Simulation, build

    build.build()
    P = lbinputs.spheres(SHAPE, 5.0, 40, seed=5, min_gap=1.0)
    rho = lbinputs.mixture(SHAPE, rho_init=(0.35, 0.35), amp=0.05, seed=6)
    s = Simulation(dict(nx=64, ny=64, nz=64, n_particles=40, radius=5.0, g_br=0.08, rho_init=(0.35, 0.35),
                        fixed_particles=1, precision=precision))
    s.init_fields(0, rho, particles=P)
    m0 = s.observables()["mass"]
    done = 0
    for t in CHECKS:
        s.step(t - done)
        done = t
        ob = s.observables()
        assert ob["error"] == 0
        rel = np.abs(ob["mass"] - m0) / m0
        bound = 1e-12 if precision == "fp64" else 10.0 * math.sqrt(t) * 4 * 2.0 ** -24
        assert np.all(rel <= bound), (precision, t, rel, bound)
    s.close()
