"""Mass correction of refilled nodes (Sec. 4, Eq. masscorr) on the CUDA path,
in the setting of the paper's long-run drift measurement (Sec. 4): moving
spheres cover and uncover nodes every step, each refill takes the mean
density of its fluid neighbours, and without a correction the total mass
of each component drifts.  With C0 > 0 every refill is scaled by
1 - C0 (sum_c' rho_init^c' / rho_init^c) dM^c / N, a proportional
controller on the drift dM^c, so the drift must stay well below the
uncorrected run's over the same steps.

Setup: 64^3, 50:50 of total density 0.7, alpha = 0.15, R = 5, neutral
wetting, particle density 3, seed 2; 4000 steps.  The flow is chaotic and
the kernels' floating-point reductions are unordered, so the drift of one
run differs from the next by tens of percent.  Over five runs on GB300s
C0 = 0 drifted by -2.3e-3 to -3.0e-3 (red) and -3.1e-3 to -3.8e-3 (blue);
C0 = 10 kept 0.29 to 0.49 (red) and 0.38 to 0.67 (blue) of that, C0 = 20
kept 0.16 to 0.31.  The test takes C0 = 20, whose reduction stays clear
of the 60 % bound from run to run."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

BOX = dict(nx=64, ny=64, nz=64, n_particles=-1, volume_fraction=0.15, radius=5.0, rho_init=(0.35, 0.35),
           contact_angle_deg=90.0, tau=(1.0, 1.0), g_br=0.08, rho0=1.0, sc_weight=(2.0, 1.0), noise_amp=0.01,
           particle_density=3.0, k_hertz=100.0, precision="fp32")


def drift(c0, steps=4000):
    from paper_1004_4414_gb300 import Simulation

    sim = Simulation([dict(BOX, mass_corr_c0=c0)])
    sim.init_from_seed(2)
    m0 = sim.observables()["mass"]
    sim.step(steps)
    ob = sim.observables()
    sim.close()
    assert ob["error"] == 0
    assert ob["n_cover"] + ob["n_uncover"] > 10_000
    return (ob["mass"] - m0) / m0


def test_mass_correction_reduces_the_drift():
    from paper_1004_4414_gb300 import build

    build.build()
    d0, d20 = drift(0.0), drift(20.0)
    # the uncorrected drift is a loss well above FP32 rounding (~1e-6)
    assert np.all(d0 < -1e-4), d0
    # the controller keeps at most 60 % of the magnitude
    assert np.all(np.abs(d20) < 0.6 * np.abs(d0)), (d0, d20)
