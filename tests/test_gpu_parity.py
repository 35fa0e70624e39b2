"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Both sides start from the same seeded inputs (lbinputs) and are compared
element by element: populations, node owners (bit-exact), particle state.
FP64 mode must agree to rounding (1e-12 absolute on populations of order
0.05, a few hundred steps); FP32 within 1e-5 relative after 100 steps on a
non-chaotic case; 16-bit deviation storage within the tolerance derived in
the test from its unit roundoff.
"""
import numpy as np
import pytest

import lbinputs
from oracle import ref

pytestmark = pytest.mark.gpu

GPU_ONLY = ("precision", "contact_angle_deg")
ORACLE_ONLY = ("virtual_fluid", "seed")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1004_4414_gb300 import build

    build.build()
    ref.lib()


def pair(precision="fp64", **params):
    from paper_1004_4414_gb300 import Simulation

    o = ref.Oracle(**{k: v for k, v in params.items() if k not in GPU_ONLY})
    s = Simulation(dict({k: v for k, v in params.items() if k not in ORACLE_ONLY}, precision=precision))
    return o, s


def compare(o, s, box=0, ftol=1e-12, ptol=1e-12, rel=False):
    a, b = s.export_state(box), o.get_state()
    assert np.array_equal(a["owner"], b["owner"]), "owners differ at %d nodes" % np.sum(a["owner"] != b["owner"])
    if rel:
        scale = np.maximum(np.abs(b["f"]), 1e-3)
        err = np.max(np.abs(a["f"] - b["f"]) / scale)
    else:
        err = np.max(np.abs(a["f"] - b["f"]))
    assert err < ftol, "populations differ by %g" % err
    if b["particles"].size:
        perr = np.max(np.abs(a["particles"] - b["particles"]))
        assert perr < ptol, "particles differ by %g" % perr
    assert a["meta"][0] == b["meta"][0]
    return err


@pytest.mark.parametrize("shape", [(16, 12, 10), (40, 9, 7), (8, 8, 8), (33, 17, 5)])
@pytest.mark.parametrize("steps", [1, 2, 7])
def test_fluid_only_fp64(shape, steps):
    """Two-component Shan-Chen fluid without particles; ragged tiles, both
    AA parities, boxes smaller than a tile (periodic wrap inside one CTA)."""
    nx, ny, nz = shape
    o, s = pair(nx=nx, ny=ny, nz=nz, n_particles=0, g_br=0.15, tau=(1.0, 0.8))
    rho = lbinputs.mixture(shape, amp=0.05, seed=1)
    o.init_fields(rho)
    s.init_fields(0, rho)
    compare(o, s)
    o.step(steps)
    s.step(steps)
    compare(o, s)


@pytest.mark.parametrize("vel_mode", [0, 1])
def test_fluid_with_velocity_field_and_body_force(vel_mode):
    shape = (20, 16, 12)
    nx, ny, nz = shape
    o, s = pair(nx=nx, ny=ny, nz=nz, n_particles=0, g_br=0.1, vel_mode=vel_mode, body_force=(1e-5, -2e-5, 0.0))
    rho = lbinputs.mixture(shape, amp=0.05, seed=3)
    u = 0.02 * np.random.default_rng(4).standard_normal((3, nx * ny * nz))
    o.init_fields(rho, u=u)
    s.init_fields(0, rho, u=u)
    o.step(9)
    s.step(9)
    compare(o, s)


@pytest.mark.parametrize("steps", [1, 4, 11])
def test_static_particles_fp64(steps):
    """Fixed spheres: bounce-back, shell virtual fluid with colour, Shan-Chen
    force on the particles."""
    shape = (24, 20, 18)
    nx, ny, nz = shape
    P = lbinputs.spheres(shape, 3.5, 3, seed=7, min_gap=1.0, vmax=0.02, wmax=0.01)
    o, s = pair(nx=nx, ny=ny, nz=nz, n_particles=3, radius=3.5, g_br=0.12, color=0.04, fixed_particles=1)
    rho = lbinputs.mixture(shape, amp=0.05, seed=8)
    o.init_fields(rho, particles=P)
    s.init_fields(0, rho, particles=P)
    o.step(steps)
    s.step(steps)
    compare(o, s)
    Fo, To = o.particle_forces()
    Fs, Ts = s.particle_forces()
    assert np.max(np.abs(Fo - Fs)) < 1e-10 and np.max(np.abs(To - Ts)) < 1e-9


@pytest.mark.parametrize("vel_mode,c0", [(0, 0.0), (1, 5.0)])
def test_moving_particles_with_events_fp64(vel_mode, c0):
    """Moving, rotating spheres: cover / uncover on both AA parities,
    momentum exchange, MD with Hertz and lubrication, optional mass
    correction; owners must match bit for bit."""
    shape = (26, 22, 20)
    nx, ny, nz = shape
    P = lbinputs.spheres(shape, 3.3, 5, seed=12, min_gap=0.4, vmax=0.06, wmax=0.03)
    o, s = pair(nx=nx, ny=ny, nz=nz, n_particles=5, radius=3.3, g_br=0.12, color=-0.03,
                particle_density=3.0, vel_mode=vel_mode, mass_corr_c0=c0)
    rho = lbinputs.mixture(shape, amp=0.05, seed=13)
    o.init_fields(rho, particles=P)
    s.init_fields(0, rho, particles=P)
    for k in range(6):
        o.step(5)
        s.step(5)
        compare(o, s, ftol=1e-11, ptol=1e-11)
    ob, sb = o.observe(), s.observables()
    assert ob["n_cover"] > 0 and ob["n_uncover"] > 0
    assert (ob["n_cover"], ob["n_uncover"]) == (sb["n_cover"], sb["n_uncover"])
    assert np.allclose(ob["mass"], sb["mass"], rtol=1e-13)
    assert np.allclose(ob["mom_fluid"] + ob["mom_part"], sb["mom_fluid"] + sb["mom_part"], atol=1e-10)


@pytest.mark.parametrize("radius", [7.6, 9.6])
def test_large_spheres_shell_rebuild_fp64(radius):
    """Large moving, rotating spheres.  R = 7.6 rebuilds its shell lists
    from the shared-memory copy of the window's flags (about 180 of a warp
    queue's 256 entries used: the surface area of a sphere is spread evenly
    over z); R = 9.6 has a window too large for that copy and takes the
    two-pass scan.  Both must give the oracle's owners, virtual densities
    and forces."""
    shape = (56, 52, 48)
    nx, ny, nz = shape
    # surface speeds up to about 0.12 (the fluid's max |u| stays below 0.16)
    P = lbinputs.spheres(shape, radius, 3, seed=41, min_gap=0.3, vmax=0.04, wmax=0.008)
    o, s = pair(nx=nx, ny=ny, nz=nz, n_particles=3, radius=radius, g_br=0.1, color=0.03, particle_density=2.0)
    rho = lbinputs.mixture(shape, amp=0.03, seed=42)
    o.init_fields(rho, particles=P)
    s.init_fields(0, rho, particles=P)
    for k in range(4):
        o.step(4)
        s.step(4)
        compare(o, s, ftol=1e-11, ptol=1e-11)
    ob, sb = o.observe(), s.observables()
    assert ob["n_cover"] > 0 and ob["n_uncover"] > 0
    assert (ob["n_cover"], ob["n_uncover"]) == (sb["n_cover"], sb["n_uncover"])


def test_many_moving_spheres_remap_fp64():
    """A box large enough for the remap's annulus scan (particles far from
    all others scan only the nodes near their surface): 36 moving, rotating
    spheres, some placed almost in contact so that particles switch between
    the annulus scan and the full window scan.  Owners stay bit-exact with
    the oracle's plain claims at every check, and the event counts agree."""
    shape = (44, 40, 36)
    nx, ny, nz = shape
    P = lbinputs.spheres(shape, 3.5, 36, seed=31, min_gap=0.15, vmax=0.08, wmax=0.04)
    o, s = pair(nx=nx, ny=ny, nz=nz, n_particles=36, radius=3.5, g_br=0.1, color=0.02, particle_density=2.0)
    rho = lbinputs.mixture(shape, amp=0.03, seed=32)
    o.init_fields(rho, particles=P)
    s.init_fields(0, rho, particles=P)
    for k in range(5):
        o.step(8)
        s.step(8)
        compare(o, s, ftol=1e-11, ptol=1e-11)
    ob, sb = o.observe(), s.observables()
    assert ob["n_cover"] > 50 and ob["n_uncover"] > 50
    assert (ob["n_cover"], ob["n_uncover"]) == (sb["n_cover"], sb["n_uncover"])


@pytest.mark.parametrize("vel_mode,c0", [(0, 0.0), (1, 5.0)])
def test_implicit_update_fp64(vel_mode, c0):
    """The implicit particle velocity update (a reading of the cited particle
    method, flag implicit_update): the drag tensor summed over the links,
    the 6 x 6 solve per particle and the fluid's share of the wall term of
    the velocity change, against the oracle, with light spheres (density 1)
    that move, rotate, cover and uncover nodes.  Fluid plus particle momentum
    stays exact."""
    shape = (26, 22, 20)
    nx, ny, nz = shape
    P = lbinputs.spheres(shape, 3.3, 5, seed=12, min_gap=0.4, vmax=0.06, wmax=0.03)
    o, s = pair(nx=nx, ny=ny, nz=nz, n_particles=5, radius=3.3, g_br=0.12, color=-0.03,
                particle_density=1.0, vel_mode=vel_mode, mass_corr_c0=c0, implicit_update=1)
    rho = lbinputs.mixture(shape, amp=0.05, seed=13)
    o.init_fields(rho, particles=P)
    s.init_fields(0, rho, particles=P)
    ob0 = s.observables()
    p0 = ob0["mom_fluid"] + ob0["mom_part"]
    for k in range(6):
        o.step(5)
        s.step(5)
        compare(o, s, ftol=1e-11, ptol=1e-11)
    ob, sb = o.observe(), s.observables()
    assert ob["n_cover"] > 0 and ob["n_uncover"] > 0
    assert (ob["n_cover"], ob["n_uncover"]) == (sb["n_cover"], sb["n_uncover"])
    p1 = sb["mom_fluid"] + sb["mom_part"]
    assert np.all(np.abs(p1 - p0) < 1e-11 * sb["mass"].sum())


@pytest.mark.parametrize("split", [0, 1])
def test_implicit_update_fp32_kernels(split):
    """Both fused kernels in FP32 with the implicit update against the FP64
    oracle on a non-chaotic case (one sphere in a mixture at g below the
    spinodal), 40 steps: populations within 1e-5 relative."""
    shape = (32, 24, 20)
    nx, ny, nz = shape
    P = lbinputs.spheres(shape, 4.0, 1, seed=3, vmax=0.02, wmax=0.01)
    o, s = pair("fp32", nx=nx, ny=ny, nz=nz, n_particles=1, radius=4.0, g_br=0.05, color=0.02,
                particle_density=1.0, implicit_update=1)
    s.set_tiling(8, 8, split)
    rho = lbinputs.mixture(shape, amp=0.01, seed=4)
    o.init_fields(rho, particles=P)
    s.init_fields(0, rho, particles=P)
    o.step(40)
    s.step(40)
    compare(o, s, ftol=1e-5, ptol=1e-5, rel=True)


def test_colors_per_particle_fp64():
    shape = (24, 24, 16)
    P = lbinputs.spheres(shape, 3.0, 4, seed=21, min_gap=1.0, vmax=0.03)
    o, s = pair(nx=24, ny=24, nz=16, n_particles=4, radius=3.0, g_br=0.15, particle_density=2.0)
    col = np.array([0.05, -0.04, 0.0, 0.02])
    rho = lbinputs.lamellae(shape, axis=2, rho_major=0.7, rho_minor=0.05)
    o.init_fields(rho, particles=P)
    s.init_fields(0, rho, particles=P)
    # initialisation gives every particle the box colour; per-particle
    # colours are set afterwards
    o.set_colors(col)
    s.set_colors(0, col)
    o.step(13)
    s.step(13)
    compare(o, s, ftol=1e-11, ptol=1e-11)


def test_seeded_init_matches_oracle():
    """lb_init_from_seed and the oracle's seeded init implement the same
    SplitMix64 streams and random sequential addition independently."""
    params = dict(nx=32, ny=32, nz=32, n_particles=16, radius=4.0, noise_amp=0.01, rho_init=(0.7, 0.7))
    o, s = pair(**params)
    o.init_from_seed(1)
    s.init_from_seed(1)
    a, b = s.export_state(), o.get_state()
    assert np.array_equal(a["particles"], b["particles"])
    assert np.array_equal(a["owner"], b["owner"])
    assert np.max(np.abs(a["f"] - b["f"])) < 1e-15


def test_config1_32cube_200_steps_fp64():
    """32^3, two components 0.7 / 0.7 with seeded noise, g = 0.08, 16 spheres
    R = 4 at random non-overlapping positions, neutral wetting, 200 steps of
    the FP64 method (particle density 2, i.e. 1.43 times the fluid density as
    in the paper's runs)."""
    params = dict(nx=32, ny=32, nz=32, n_particles=16, radius=4.0, noise_amp=0.01, rho_init=(0.7, 0.7),
                  g_br=0.08, particle_density=2.0)
    o, s = pair(**params)
    o.init_from_seed(1)
    s.init_from_seed(1)
    for k in range(4):
        o.step(50)
        s.step(50)
        compare(o, s, ftol=1e-10, ptol=1e-10)
    sb = s.observables()
    assert sb["error"] == 0 and sb["n_cover"] > 0


def test_import_export_roundtrip_and_odd_parity():
    """A state exported by the oracle at an odd step is imported into the
    GPU (AA odd-parity layout) and stepped on.  Export returns the moving
    populations exactly.  The GPU keeps rho^c, not f_0: import sums the 19
    populations into the density and export gives f_0 back as rho^c minus
    the 18 moving ones, so f_0 returns to within the rounding of those two
    sums (19 additions of values below 1 in FP64)."""
    shape = (22, 18, 14)
    nx, ny, nz = shape
    P = lbinputs.spheres(shape, 3.0, 3, seed=31, min_gap=0.5, vmax=0.05, wmax=0.02)
    o, s = pair(nx=nx, ny=ny, nz=nz, n_particles=3, radius=3.0, g_br=0.12, color=0.02, particle_density=2.5)
    o.init_fields(lbinputs.mixture(shape, amp=0.05, seed=32), particles=P)
    o.step(7)
    st = o.get_state()
    s.import_state(0, st)
    back = s.export_state(0)
    f_in = np.asarray(st["f"]).reshape(2, 19, -1)
    assert np.array_equal(back["f"][:, 1:], f_in[:, 1:]) and np.array_equal(back["owner"], st["owner"])
    assert np.max(np.abs(back["f"][:, 0] - f_in[:, 0])) <= 64 * 2.0 ** -53
    assert np.array_equal(back["particles"], st["particles"])
    o.step(9)
    s.step(9)
    compare(o, s, ftol=1e-11, ptol=1e-11)


def test_walls_poiseuille_fp64():
    nz = 18
    walls = np.full((nz, 4, 3), -1, np.int32)
    walls[0] = walls[nz - 1] = -2
    o, s = pair(nx=3, ny=4, nz=nz, n_particles=0, g_br=0.0, tau=(0.9, 0.9), body_force=(1e-5, 0.0, 0.0))
    rho = np.full((2, 3 * 4 * nz), 0.5)
    o.init_fields(rho, walls=walls.reshape(-1))
    s.init_fields(0, rho, walls=walls.reshape(-1))
    o.step(300)
    s.step(300)
    compare(o, s)


@pytest.mark.parametrize("ty,cz", [(4, 3), (8, 1), (16, 5), (8, 64)])
def test_tilings_agree(ty, cz):
    shape = (37, 29, 23)
    nx, ny, nz = shape
    P = lbinputs.spheres(shape, 3.5, 4, seed=41, min_gap=0.5, vmax=0.04, wmax=0.02)
    o, s = pair(nx=nx, ny=ny, nz=nz, n_particles=4, radius=3.5, g_br=0.12, color=0.03, particle_density=2.0)
    s.set_tiling(ty, cz)
    rho = lbinputs.mixture(shape, amp=0.05, seed=42)
    o.init_fields(rho, particles=P)
    s.init_fields(0, rho, particles=P)
    o.step(12)
    s.step(12)
    compare(o, s, ftol=1e-11, ptol=1e-11)


def test_retiling_mid_run():
    """Changing the block shape between steps (as the autotuner does) keeps
    the state exact."""
    shape = (40, 24, 20)
    nx, ny, nz = shape
    P = lbinputs.spheres(shape, 3.5, 3, seed=43, min_gap=0.5, vmax=0.04, wmax=0.02)
    o, s = pair(nx=nx, ny=ny, nz=nz, n_particles=3, radius=3.5, g_br=0.12, color=0.03, particle_density=2.0)
    rho = lbinputs.mixture(shape, amp=0.05, seed=44)
    o.init_fields(rho, particles=P)
    s.init_fields(0, rho, particles=P)
    for ty, cz, split in ((8, 4, 0), (16, 6, 1), (4, 7, 0), (8, 20, 1), (16, 20, 0), (8, 1, 0), (4, 3, 0)):
        s.set_tiling(ty, cz, split)
        s.step(3)
        o.step(3)
    compare(o, s, ftol=1e-11, ptol=1e-11)
    assert s.observables()["error"] == 0


# ------------------------------------- one thread per node and component
@pytest.mark.parametrize("ty,cz", [(8, 1), (16, 5), (8, 64), (16, 3)])
def test_split_kernel_moving_particles(ty, cz):
    """The kernel with the two components on the two halves of a warp
    (16-wide tiles; 37 = 16 + 16 + 5 leaves a ragged tile) against the
    oracle, with moving spheres and cover / uncover events."""
    shape = (37, 29, 23)
    nx, ny, nz = shape
    P = lbinputs.spheres(shape, 3.5, 4, seed=41, min_gap=0.5, vmax=0.04, wmax=0.02)
    o, s = pair(nx=nx, ny=ny, nz=nz, n_particles=4, radius=3.5, g_br=0.12, color=0.03, particle_density=2.0)
    s.set_tiling(ty, cz, 1)
    rho = lbinputs.mixture(shape, amp=0.05, seed=42)
    o.init_fields(rho, particles=P)
    s.init_fields(0, rho, particles=P)
    o.step(12)
    s.step(12)
    compare(o, s, ftol=1e-11, ptol=1e-11)


@pytest.mark.parametrize("shape", [(16, 12, 10), (40, 9, 7), (8, 8, 8), (5, 3, 4)])
def test_split_kernel_fluid_tau_not_one(shape):
    """Split kernel with tau^b != 1 (the general BGK path, not the tau = 1
    specialisation), boxes narrower than a tile and a box of 5 x 3 nodes
    where every node is a tile-edge node."""
    nx, ny, nz = shape
    o, s = pair(nx=nx, ny=ny, nz=nz, n_particles=0, g_br=0.15, tau=(1.0, 0.8))
    s.set_tiling(8, 3, 1)
    rho = lbinputs.mixture(shape, amp=0.05, seed=1)
    o.init_fields(rho)
    s.init_fields(0, rho)
    o.step(7)
    s.step(7)
    compare(o, s)


@pytest.mark.parametrize("vel_mode,c0", [(0, 0.0), (1, 5.0)])
def test_split_kernel_velocity_modes_and_mass_correction(vel_mode, c0):
    """Split kernel with both velocity definitions (the partner's moments
    enter u' only for vel_mode 0), a body force, and the mass correction."""
    shape = (26, 22, 20)
    nx, ny, nz = shape
    P = lbinputs.spheres(shape, 3.3, 5, seed=12, min_gap=0.4, vmax=0.06, wmax=0.03)
    o, s = pair(nx=nx, ny=ny, nz=nz, n_particles=5, radius=3.3, g_br=0.12, color=-0.03, tau=(0.9, 1.2),
                particle_density=3.0, vel_mode=vel_mode, mass_corr_c0=c0, body_force=(1e-5, -2e-5, 0.0))
    s.set_tiling(16, 4, 1)
    rho = lbinputs.mixture(shape, amp=0.05, seed=13)
    o.init_fields(rho, particles=P)
    s.init_fields(0, rho, particles=P)
    for k in range(4):
        o.step(5)
        s.step(5)
        compare(o, s, ftol=1e-11, ptol=1e-11)
    ob, sb = o.observe(), s.observables()
    assert ob["n_cover"] > 0 and ob["n_uncover"] > 0
    assert np.allclose(ob["mass"], sb["mass"], rtol=1e-13)


def test_long_y_axis_beyond_16_bit_signed():
    """Node coordinates are packed as x | y << 16 in the shell lists; a box
    with y up to 32809 puts a moving, rotating sphere across y = 32767 so that
    its shell nodes carry y >= 2^15 (read back unsigned)."""
    shape = (12, 32810, 12)
    nx, ny, nz = shape
    P = np.zeros((1, 9))
    P[0, 0:3] = (5.6, 32767.3, 6.2)
    P[0, 3:6] = (0.01, 0.03, -0.02)
    P[0, 6:9] = (0.0, 0.02, 0.01)
    o, s = pair(nx=nx, ny=ny, nz=nz, n_particles=1, radius=3.2, g_br=0.1, color=0.03, particle_density=2.0)
    rho = lbinputs.mixture(shape, amp=0.05, seed=51)
    o.init_fields(rho, particles=P)
    s.init_fields(0, rho, particles=P)
    o.step(4)
    s.step(4)
    compare(o, s, ftol=1e-11, ptol=1e-11)
    Fo, To = o.particle_forces()
    Fs, Ts = s.particle_forces()
    assert np.max(np.abs(Fo - Fs)) < 1e-9 and np.max(np.abs(To - Ts)) < 1e-9


def test_batched_boxes_fp64():
    """Uneven boxes stepped together in one launch per phase."""
    from paper_1004_4414_gb300 import Simulation

    specs = [dict(nx=16, ny=16, nz=16, n_particles=2, radius=3.0, color=0.03),
             dict(nx=24, ny=20, nz=12, n_particles=3, radius=2.5, color=-0.02, g_br=0.1),
             dict(nx=12, ny=12, nz=20, n_particles=0)]
    s = Simulation([dict(sp, precision="fp64", particle_density=2.0) for sp in specs])
    oracles = []
    for b, sp in enumerate(specs):
        shape = (sp["nx"], sp["ny"], sp["nz"])
        P = lbinputs.spheres(shape, sp.get("radius", 5.0), sp["n_particles"], seed=50 + b, min_gap=0.5,
                             vmax=0.04, wmax=0.02) if sp["n_particles"] else None
        rho = lbinputs.mixture(shape, amp=0.04, seed=60 + b)
        o = ref.Oracle(**dict(sp, particle_density=2.0))
        o.init_fields(rho, particles=P)
        s.init_fields(b, rho, particles=P)
        oracles.append(o)
    for o in oracles:
        o.step(10)
    s.step(10)
    for b, o in enumerate(oracles):
        compare(o, s, box=b, ftol=1e-11, ptol=1e-11)


# ------------------------------------------------------------------- FP32
@pytest.mark.parametrize("split", [0, 1])
def test_fp32_non_chaotic_100_steps(split):
    """FP32 populations within 1e-5 relative of FP64 after 100 steps on a
    non-chaotic case (a lamella with a resting particle, below the spinodal
    coupling), with both fused kernels."""
    shape = (32, 24, 20)
    nx, ny, nz = shape
    P = np.zeros((1, 9))
    P[0, 0:3] = (15.3, 11.7, 9.6)
    o, s = pair("fp32", nx=nx, ny=ny, nz=nz, n_particles=1, radius=4.0, g_br=0.05, color=0.02,
                fixed_particles=1)
    s.set_tiling(8, 32, split)
    rho = lbinputs.lamellae(shape, axis=2, rho_major=0.6, rho_minor=0.3)
    o.init_fields(rho, particles=P)
    s.init_fields(0, rho, particles=P)
    o.step(100)
    s.step(100)
    compare(o, s, ftol=1e-5, rel=True)


def test_fp32_mass_conserved():
    shape = (48, 40, 36)
    P = lbinputs.spheres(shape, 4.0, 6, seed=71, min_gap=1.0)
    from paper_1004_4414_gb300 import Simulation

    s = Simulation(dict(nx=48, ny=40, nz=36, n_particles=6, radius=4.0, g_br=0.1, color=0.03,
                        fixed_particles=1, precision="fp32"))
    s.init_fields(0, lbinputs.mixture(shape, amp=0.05, seed=72), particles=P)
    m0 = s.observables()["mass"]
    s.step(200)
    ob = s.observables()
    assert ob["error"] == 0
    assert np.all(np.abs(ob["mass"] - m0) / m0 < 1e-6)


@pytest.mark.parametrize("split", [0, 1])
@pytest.mark.parametrize("prec,eps", [("fp16", 2.0 ** -11), ("bf16", 2.0 ** -8)])
def test_deviation_storage(prec, eps, split):
    """16-bit deviation storage: each stored population carries a relative
    error of at most the unit roundoff u of its deviation d = f/zeta - rho_ref,
    so a population deviates by <= zeta |d| u per step; the rest population
    (the FP32 density minus the 18 stored values) absorbs the 16-bit
    rounding, so mass is conserved up to FP32
    rounding."""
    shape = (32, 24, 20)
    nx, ny, nz = shape
    P = np.zeros((1, 9))
    P[0, 0:3] = (15.3, 11.7, 9.6)
    o, s = pair(prec, nx=nx, ny=ny, nz=nz, n_particles=1, radius=4.0, g_br=0.05, color=0.02,
                fixed_particles=1, rho_init=(0.45, 0.45))
    s.set_tiling(8, 32, split)
    rho = lbinputs.lamellae(shape, axis=2, rho_major=0.6, rho_minor=0.3)
    o.init_fields(rho, particles=P)
    s.init_fields(0, rho, particles=P)
    m0 = s.observables()["mass"]
    steps = 50
    o.step(steps)
    s.step(steps)
    a, b = s.export_state(), o.get_state()
    assert np.array_equal(a["owner"], b["owner"])
    # |d| <= 0.6 here; errors of successive steps are damped by BGK (tau = 1
    # replaces f by f^eq of the local moments), so the bound is a few roundoffs
    tol = 8 * 0.6 * eps * (1.0 / 18)
    err = np.max(np.abs(a["f"] - b["f"]))
    assert err < tol, (err, tol)
    ob = s.observables()
    # mass: per node and step, the 18 reconstructions zeta (rho_ref + d) and
    # the roundings of the rest population and of the FP32 density sum add a
    # few 2^-24 rho; on this layered state identical nodes round alike, so
    # the worst case adds up coherently over the 50 steps
    assert np.all(np.abs(ob["mass"] - m0) / m0 < steps * 4 * 2.0 ** -24)


# --------------------------------------------------------------- spheroids
@pytest.mark.parametrize("aspect", [1.75, 0.6])
def test_spheroid_seeded_init_matches_oracle(aspect):
    """Seeded spheroids (semi-axes R, R, aspect R): the same axes from stream
    3, the same placement and bit-identical node owners."""
    params = dict(nx=36, ny=36, nz=36, n_particles=8, radius=4.0, aspect=aspect, noise_amp=0.01)
    o, s = pair(**params)
    o.init_from_seed(3)
    s.init_from_seed(3)
    a, b = s.export_state(), o.get_state()
    assert np.array_equal(a["particles"], b["particles"])
    assert np.array_equal(s.axes(), o.axes())
    bad = s.axes().copy()
    bad[0] *= 1.01  # not a unit vector: rejected, axes unchanged
    with pytest.raises(Exception):
        s.set_axes(0, bad)
    assert np.array_equal(s.axes(), o.axes())
    assert np.array_equal(a["owner"], b["owner"])
    assert np.max(np.abs(a["f"] - b["f"])) < 1e-15


@pytest.mark.parametrize("aspect,split", [(1.75, 0), (0.6, 0), (1.75, 1)])
def test_moving_spheroids_with_events_fp64(aspect, split):
    """Moving, rotating spheroids: claims with the spheroid inside test and
    turning axes, cover / uncover on both parities, contact forces along the
    line of centres, rotation about the angular momentum; owners bit-exact,
    populations, particle state and axes to the FP64 rounding level."""
    shape = (30, 28, 32)
    nx, ny, nz = shape
    params = dict(nx=nx, ny=ny, nz=nz, n_particles=4, radius=3.5, aspect=aspect, g_br=0.12, color=0.03,
                  particle_density=3.0)
    o0 = ref.Oracle(**params)
    o0.init_from_seed(9)
    P = o0.get_state()["particles"].copy()
    E = o0.axes()
    P[:, 3:6] = [[0.05, -0.03, 0.02], [-0.04, 0.02, 0.03], [0.01, 0.05, -0.04], [0.03, 0.01, 0.04]]
    P[:, 6:9] = [[0.01, 0.02, -0.01], [0.0, -0.02, 0.015], [0.02, 0.0, 0.01], [-0.01, 0.01, 0.02]]
    o, s = pair(**params)
    if split:
        s.set_tiling(8, 5, 1)
    o.set_axes(E)
    s.set_axes(0, E)
    rho = lbinputs.mixture(shape, amp=0.05, seed=14)
    o.init_fields(rho, particles=P)
    s.init_fields(0, rho, particles=P)
    for k in range(5):
        o.step(5)
        s.step(5)
        compare(o, s, ftol=1e-11, ptol=1e-11)
        assert np.max(np.abs(s.axes() - o.axes())) < 1e-11
    ob, sb = o.observe(), s.observables()
    assert ob["n_cover"] > 0 and ob["n_uncover"] > 0
    assert (ob["n_cover"], ob["n_uncover"]) == (sb["n_cover"], sb["n_uncover"])
    assert not np.allclose(s.axes(), E)
    assert np.allclose(ob["mom_fluid"] + ob["mom_part"], sb["mom_fluid"] + sb["mom_part"], atol=1e-10)


def test_overlapping_spheroids_fp64():
    """Overlapping spheroids against the oracle, bit for bit on the owners:
    (a) deep overlap, particles held fixed: the initial claims (nearest
    centre among the spheroids a node lies in) and the remap's claims with
    the close-neighbour list; (b) a shallow overlap (0.5 along the line of
    centres, soft contact) moving apart, so nodes change hands."""
    L = 24
    E = np.array([[1.0, 0.2, 0.1], [-0.3, 1.0, 0.4]])
    E /= np.linalg.norm(E, axis=1, keepdims=True)
    base = dict(nx=L, ny=L, nz=L, n_particles=2, radius=4.0, aspect=1.75, g_br=0.1, color=0.02,
                particle_density=3.0)
    rho = lbinputs.mixture((L, L, L), amp=0.05, seed=21)
    # (a) deep overlap, fixed
    P = np.zeros((2, 9))
    P[0, :3] = (10.3, 11.6, 12.2)
    P[1, :3] = (14.1, 12.4, 11.7)
    o, s = pair(**base, fixed_particles=1)
    o.set_axes(E)
    s.set_axes(0, E)
    o.init_fields(rho, particles=P)
    s.init_fields(0, rho, particles=P)
    compare(o, s)
    o.step(4)
    s.step(4)
    compare(o, s, ftol=1e-11, ptol=1e-11)
    # (b) shallow overlap along r_hat (contact distance 10.76 for these axes), moving apart
    rh = np.array([1.0, 0.2, -0.1]) / np.linalg.norm([1.0, 0.2, -0.1])
    P = np.zeros((2, 9))
    P[0, :3] = (6.3, 11.6, 12.2)
    P[1, :3] = P[0, :3] + 10.26 * rh
    P[0, 3:6] = -0.02 * rh
    P[1, 3:6] = 0.02 * rh
    P[1, 6:9] = (0.0, 0.01, 0.005)
    o, s = pair(**base, k_hertz=1.0)
    o.set_axes(E)
    s.set_axes(0, E)
    o.init_fields(rho, particles=P)
    s.init_fields(0, rho, particles=P)
    for k in range(4):
        o.step(5)
        s.step(5)
        compare(o, s, ftol=1e-11, ptol=1e-11)
        assert np.max(np.abs(s.axes() - o.axes())) < 1e-11
    ob = o.observe()
    assert ob["n_uncover"] > 0 and ob["n_cover"] > 0


def test_import_rejects_invalid_owner_without_changes():
    """lb_import_state with an owner entry outside [-2, n_particles) returns
    LB_EINVAL before any part of the box changes."""
    shape = (16, 12, 10)
    nx, ny, nz = shape
    P = lbinputs.spheres(shape, 2.5, 2, seed=5, min_gap=1.0, vmax=0.02)
    o, s = pair(nx=nx, ny=ny, nz=nz, n_particles=2, radius=2.5, g_br=0.1)
    rho = lbinputs.mixture(shape, amp=0.05, seed=6)
    s.init_fields(0, rho, particles=P)
    s.step(3)
    before = s.export_state(0)
    bad = dict(before, owner=before["owner"].copy(), particles=before["particles"] + 0.5)
    bad["owner"][7] = 5  # no particle 5 in this box
    with pytest.raises(Exception):
        s.import_state(0, bad)
    after = s.export_state(0)
    assert np.array_equal(after["owner"], before["owner"])
    assert np.array_equal(after["particles"], before["particles"])
    assert np.array_equal(after["f"], before["f"])
