"""The CUDA path at the full sizes of the benchmark workloads, in the launch
configuration bench.py times (autotuned tiling, FP32), against the FP64
oracle on sampled outputs, and through properties that hold at any size.

The 256^3 parameters are those of bench.py's c256 workload: fluid ratio
60:40 of total density 0.7 (0.42 / 0.28), alpha = 0.20, R = 5, contact
angle 77 deg (colour (77 - 90) / 442), g = 0.08, particle density 3,
seed 3 (6408 spheres)."""
import os

import numpy as np
import pytest

from oracle import ref

pytestmark = pytest.mark.gpu

C256 = dict(nx=256, ny=256, nz=256, n_particles=-1, tau=(1.0, 1.0), g_br=0.08, rho0=1.0, sc_weight=(2.0, 1.0),
            rho_init=(0.42, 0.28), noise_amp=0.01, volume_fraction=0.20, radius=5.0, particle_density=3.0,
            k_hertz=100.0)
COLOR_77 = (77.0 - 90.0) / 442.0
SEED = 3


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1004_4414_gb300 import build

    build.build()
    ref.lib()
    ref.set_threads(os.cpu_count() or 1)


def _sim(**kw):
    from paper_1004_4414_gb300 import Simulation

    return Simulation(dict(C256, contact_angle_deg=77.0, **kw))


def test_c256_two_steps_sampled_against_oracle():
    """Two steps (an even and an odd AA step) of the 256^3 workload with the
    tiling the benchmark uses: node owners bit-exact everywhere, FP32
    populations within 1e-5 relative of FP64 on 200,000 sampled nodes, and
    the particle state after the MD update."""
    from paper_1004_4414_gb300.autotune import autotune

    sim = _sim(precision="fp32")
    sim.init_from_seed(SEED)
    autotune(sim)  # as bench.py: tune on the seeded state, then start again
    sim.init_from_seed(SEED)
    o = ref.Oracle(**C256, color=COLOR_77)
    o.init_from_seed(SEED)
    assert o.np == sim.n_particles[0] == 6408
    sim.step(2)
    o.step(2)
    a, b = sim.export_state(0), o.get_state()
    sim.close()
    assert np.array_equal(a["owner"], b["owner"])
    idx = np.random.default_rng(0).choice(b["owner"].size, 200_000, replace=False)
    fa, fb = a["f"][:, :, idx], b["f"][:, :, idx]
    err = np.max(np.abs(fa - fb) / np.maximum(np.abs(fb), 1e-3))
    assert err < 1e-5, err
    # MD in FP64 from FP32 force sums: a particle's force adds ~2000 link
    # terms of magnitude <= 0.1 in FP32, worst case 2000 * 0.1 * 6e-8 = 1.2e-5
    # per step, i.e. <= 7.6e-9 in U (m = 3 * 4/3 pi 125 = 1571) and, after two
    # leap-frog steps, <= 2.3e-8 in X and 1.5e-8 in U (omega: J = 2/5 m R^2)
    assert np.max(np.abs(a["particles"][:, :3] - b["particles"][:, :3])) < 2.3e-8
    assert np.max(np.abs(a["particles"][:, 3:] - b["particles"][:, 3:])) < 1.5e-8


def test_c256_total_momentum_conserved_moving_particles():
    """Fluid plus particle momentum is conserved by every coupling term
    (momentum exchange, cover/uncover, shell force, pair forces); at 256^3
    in FP32 the change over 10 steps stays at the rounding level of the
    stored populations (a sign error in any term would exceed it by orders
    of magnitude)."""
    sim = _sim(precision="fp32")
    sim.init_from_seed(SEED)
    o0 = sim.observables()
    p0 = o0["mom_fluid"] + o0["mom_part"]
    sim.step(10)
    o1 = sim.observables()
    sim.close()
    assert o1["error"] == 0
    assert o1["n_cover"] + o1["n_uncover"] > 0
    p1 = o1["mom_fluid"] + o1["mom_part"]
    scale = o0["mass"].sum() * 0.04
    assert np.all(np.abs(p1 - p0) < 1e-7 * scale), (p1 - p0, scale)


def test_c512_fp16_mass_conserved_fixed_particles():
    """The largest configuration, 512^3 with 51,267 spheres (the paper's
    alpha = 0.20, R = 5) in FP16 deviation storage: with the particles held
    fixed (no cover/uncover) each component's mass is conserved to the
    rounding of the FP32 density field."""
    from paper_1004_4414_gb300 import Simulation

    box = dict(C256, nx=512, ny=512, nz=512, rho_init=(0.35, 0.35), contact_angle_deg=90.0, precision="fp16",
               fixed_particles=1)
    sim = Simulation(box)
    assert sim.n_particles[0] == 51267  # round(0.2 * 512^3 / (4/3 pi 125)) = round(51267.4)
    sim.init_from_seed(5)
    m0 = sim.observables()["mass"]
    sim.step(4)
    ob = sim.observables()
    sim.close()
    assert ob["error"] == 0
    assert np.all(np.abs(ob["mass"] - m0) / m0 < 2e-6), (ob["mass"] - m0) / m0
