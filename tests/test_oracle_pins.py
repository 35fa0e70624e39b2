"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage or theory it relies on.  They are chosen so
that a plausible slip anywhere in the oracle -- a wrong weight or sign, a
dropped term, a transposed index, a force applied to the wrong particle or
component -- fails at least one of them.
"""
import itertools
import os

import numpy as np
import pytest

import lbinputs
from oracle import analysis as oan
from oracle import ref

CS2 = 1.0 / 3.0
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- lattice
def test_lattice_isotropy():
    """D3Q19 (Sec. II): weights sum to 1; second and fourth moments are
    isotropic with c_s^2 = 1/3 (textbook lattice conditions)."""
    c, w, opp = ref.lattice()
    c = c.astype(np.float64)
    assert abs(w.sum() - 1.0) < 1e-15
    M2 = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.allclose(M2, CS2 * np.eye(3), atol=1e-15)
    M4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(3)
    iso = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                      + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(M4, iso, atol=1e-15)
    for i in range(19):
        assert np.all(c[opp[i]] == -c[i])
    assert sorted(map(tuple, c.astype(int))) == sorted(
        {v for v in itertools.product((-1, 0, 1), repeat=3) if sum(map(abs, v)) <= 2})


def _feq_hermite(rho, u, c, w):
    """Third-order Hermite expansion of the Maxwellian on the lattice built
    from the tensor Hermite polynomials H0..H3 (an independent construction
    of Eq. Equil)."""
    c = c.astype(np.float64)
    d = np.eye(3)
    out = np.zeros(19)
    for i in range(19):
        ci = c[i]
        H1 = ci
        H2 = np.outer(ci, ci) - CS2 * d
        H3 = np.einsum("a,b,c->abc", ci, ci, ci) - CS2 * (
            np.einsum("a,bc->abc", ci, d) + np.einsum("b,ac->abc", ci, d) + np.einsum("c,ab->abc", ci, d))
        a1 = u
        a2 = np.outer(u, u)
        a3 = np.einsum("a,b,c->abc", u, u, u)
        out[i] = w[i] * rho * (1.0 + np.dot(H1, a1) / CS2 + np.sum(H2 * a2) / (2 * CS2 ** 2)
                               + np.sum(H3 * a3) / (6 * CS2 ** 3))
    return out


def test_feq_is_third_order_hermite():
    c, w, _ = ref.lattice()
    rng = np.random.default_rng(3)
    for _ in range(20):
        rho = 0.2 + rng.random()
        u = 0.2 * (rng.random(3) - 0.5)
        assert np.allclose(ref.feq(rho, u), _feq_hermite(rho, u, c, w), rtol=0, atol=1e-15)


def test_feq_moments():
    """Mass and momentum of Eq. Equil are exact (the cubic terms cancel in the
    first moment because the D3Q19 fourth moment is isotropic); the second
    moment is rho (c_s^2 I + u u)."""
    c, w, _ = ref.lattice()
    c = c.astype(np.float64)
    rng = np.random.default_rng(1)
    for _ in range(20):
        rho = 0.1 + rng.random()
        u = 0.3 * (rng.random(3) - 0.5)
        f = ref.feq(rho, u)
        assert abs(f.sum() - rho) < 1e-15
        assert np.allclose(f @ c, rho * u, atol=1e-16)
        assert np.allclose(np.einsum("i,ia,ib->ab", f, c, c), rho * (CS2 * np.eye(3) + np.outer(u, u)), atol=1e-15)


def test_splitmix64_reference_vector():
    vals = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt")) if l.strip() and not l.startswith("#")]
    assert [ref.splitmix64(1234567, k) for k in range(5)] == vals
    u = [ref.unit(1234567, k) for k in range(5)]
    assert u == [(v >> 11) / 2.0 ** 53 for v in vals]


# ----------------------------------------------------------- conservation
def _total_momentum(o):
    ob = o.observe()
    return ob["mom_fluid"] + ob["mom_part"]


def test_mass_conserved_without_particles():
    """BGK collision and periodic streaming conserve each component's mass
    (Eq. eq:boltz; Sigma_i f^eq = rho)."""
    shape = (12, 10, 8)
    o = ref.Oracle(nx=12, ny=10, nz=8, n_particles=0, g_br=0.2, tau=(1.0, 0.8))
    o.init_fields(lbinputs.mixture(shape, amp=0.05, seed=2))
    m0 = o.observe()["mass"]
    o.step(60)
    m1 = o.observe()["mass"]
    assert np.all(np.abs(m1 - m0) / m0 < 1e-13)
    # and no net momentum appears from the pairwise Shan-Chen force
    assert np.all(np.abs(o.observe()["mom_fluid"]) < 1e-12)


def test_mass_conserved_static_particles():
    """Bounce-back returns every population to the fluid (Eq. eqn_bounce-back):
    resting, fixed spheres conserve each component's mass exactly."""
    shape = (16, 16, 16)
    P = lbinputs.spheres(shape, 3.0, 3, seed=5, min_gap=1.0)
    o = ref.Oracle(nx=16, ny=16, nz=16, n_particles=3, radius=3.0, g_br=0.12, color=0.03,
                   fixed_particles=1)
    o.init_fields(lbinputs.mixture(shape, amp=0.05, seed=3), particles=P)
    m0 = o.observe()["mass"]
    o.step(40)
    m1 = o.observe()["mass"]
    assert np.all(np.abs(m1 - m0) / m0 < 1e-13)


@pytest.mark.parametrize("vel_mode", [0, 1])
def test_total_momentum_conserved_with_moving_particles(vel_mode):
    """Fluid + particle momentum is conserved exactly when every particle
    force carries the sign that balances the fluid's change: momentum
    exchange (Eq. eqn_ladd_bewegtewand), cover / uncover
    (Eq. eqn_ladd_vernichtenunderzeugen), the shell Shan-Chen force
    (Eq. eqn_shan_chen_particle) and the pairwise MD forces."""
    shape = (20, 18, 16)
    P = lbinputs.spheres(shape, 3.2, 4, seed=11, min_gap=0.3, vmax=0.04, wmax=0.02)
    o = ref.Oracle(nx=20, ny=18, nz=16, n_particles=4, radius=3.2, g_br=0.15, color=0.04,
                   particle_density=3.0, vel_mode=vel_mode, mass_corr_c0=5.0)
    o.set_colors(np.array([0.04, -0.03, 0.0, 0.05]))
    o.init_fields(lbinputs.mixture(shape, amp=0.05, seed=12), particles=P)
    p0 = _total_momentum(o)
    scale = o.observe()["mass"].sum() * 0.04
    o.step(60)
    ob = o.observe()
    assert ob["n_cover"] > 0 and ob["n_uncover"] > 0
    p1 = _total_momentum(o)
    assert np.all(np.abs(p1 - p0) < 1e-11 * scale)


def test_momentum_balance_detects_wrong_sign():
    """Control for the test above: the particle momentum alone changes, so
    conservation is not trivially satisfied."""
    shape = (20, 18, 16)
    P = lbinputs.spheres(shape, 3.2, 4, seed=11, min_gap=0.3, vmax=0.04, wmax=0.02)
    o = ref.Oracle(nx=20, ny=18, nz=16, n_particles=4, radius=3.2, g_br=0.15, color=0.04,
                   particle_density=3.0)
    o.init_fields(lbinputs.mixture(shape, amp=0.05, seed=12), particles=P)
    mp0 = o.observe()["mom_part"].copy()
    o.step(20)
    mp1 = o.observe()["mom_part"]
    assert np.max(np.abs(mp1 - mp0)) > 1e-3


# -------------------------------------------------- Shan-Chen force stencil
def _wave_growth(g, weights, tau, steps=3000, rho_bar=0.7, n=32):
    """Amplitude ratio of a small antisymmetric composition wave."""
    x = np.arange(n)
    eps = 1e-4
    dr = eps * np.sin(2 * np.pi * x / n)
    rho = np.stack([rho_bar + dr, rho_bar - dr])
    o = ref.Oracle(nx=n, ny=1, nz=1, n_particles=0, g_br=g, sc_weight=weights, tau=(tau, tau))
    o.init_fields(rho)
    o.step(steps)
    r = o.rho()
    phi = r[0] - r[1]
    amp = 2 * abs(np.sum(phi * np.sin(2 * np.pi * x / n))) / n
    return amp / (2 * eps)


@pytest.mark.parametrize("weights,A,tau", [((1.0, 1.0), 10.0, 1.0), ((2.0, 1.0), 12.0, 1.0),
                                           ((2.0, 1.0), 12.0, 0.8)])
def test_spinodal_threshold(weights, A, tau):
    """Linear stability of the scheme of Sec. II about a 50:50 mixture.  The
    velocity shift tau F / rho makes the composition flux of a component
    tau F^c - c_s^2 (tau - 1/2) grad rho^c, and linearising
    Eq. eqn_shan-chen-F with Eq. eqn_ref_dens gives F^r = g A Psi Psi' grad
    (rho^r - rho_bar), A = sum_i W_i c_ix^2, Psi' = exp(-rho/rho0).  A long
    wave therefore grows iff tau g A Psi Psi' > c_s^2 (tau - 1/2).  Bracketing
    the threshold at +-5% pins the force sign, the Psi form, the split of the
    link weights between axis and diagonal links, and the velocity shift
    (the tau dependence).  The long-wave threshold lies 1% above the formula
    at this wavelength (k = 2 pi / 32), inside the bracket."""
    rho = 0.7
    pp = (1.0 - np.exp(-rho)) * np.exp(-rho)
    gc = CS2 * (tau - 0.5) / (tau * A * pp)
    assert _wave_growth(1.05 * gc, weights, tau) > 1.0
    assert _wave_growth(0.95 * gc, weights, tau) < 1.0


# ------------------------------------------------------------ bounce-back
def test_poiseuille_magic_tau():
    """Plane Poiseuille flow between static bounce-back walls (Eq.
    eqn_bounce-back).  The BGK solution is a parabola with curvature -g/nu,
    nu = c_s^2 (tau - 1/2) (Sec. II), and for (tau - 1/2)^2 = 3/16 it
    vanishes exactly half-way between the last fluid and the first wall node
    (He et al., J. Stat. Phys. 87, 115 (1997); Ginzburg & d'Humieres,
    PRE 68, 066614 (2003))."""
    nz = 18
    tau = 0.5 + np.sqrt(3.0 / 16.0)
    g = 1e-6
    walls = np.full((nz, 1, 1), -1, np.int32)
    walls[0] = walls[nz - 1] = -2
    o = ref.Oracle(nx=1, ny=1, nz=nz, n_particles=0, g_br=0.0, tau=(tau, tau),
                   body_force=(g, 0.0, 0.0))
    rho = np.full((2, nz), 0.5)
    o.init_fields(rho, walls=walls.reshape(-1))
    o.step(12000)
    u = o.velocity()[0].reshape(nz)
    z = np.arange(1, nz - 1, dtype=np.float64)
    uf = u[1:nz - 1] + 0.5 * g  # physical velocity includes half the force per unit mass
    coef = np.polyfit(z, uf, 2)
    nu = CS2 * (tau - 0.5)
    assert abs(coef[0] * 2 / (-g / nu) - 1.0) < 1e-6
    roots = np.sort(np.roots(coef).real)
    assert abs(roots[0] - 0.5) < 1e-5 and abs(roots[1] - (nz - 1.5)) < 1e-5
    resid = uf - np.polyval(coef, z)
    assert np.max(np.abs(resid)) < 1e-9 * np.max(uf)


def _comoving_error(U):
    P = np.zeros((1, 9))
    P[0, 0:3] = (7.3, 8.1, 7.6)
    P[0, 3:6] = U
    o = ref.Oracle(nx=16, ny=16, nz=16, n_particles=1, radius=4.0, g_br=0.0,
                   fixed_particles=1)
    u = np.tile(np.asarray(U, float).reshape(3, 1), (1, 16 ** 3))
    o.init_fields(np.full((2, 16 ** 3), 0.6), u=u, particles=P)
    o.step(1)
    st = o.get_state()
    fluid = st["owner"] == -1
    vel = o.velocity()[:, fluid]
    mass_err = np.max(np.abs(st["f"].sum(axis=(0, 1))[fluid] - 1.2))
    return np.max(np.abs(vel - np.asarray(U, float)[:, None])), mass_err


def test_moving_wall_term_galilean():
    """A sphere moving with the surrounding uniform flow leaves it
    undisturbed up to the cubic terms of Eq. Equil: the moving-wall term
    6 zeta_j rho u_s.c_j of Eq. eqn_ladd_bewegtewand cancels the odd linear
    part of f^eq_j - f^eq_opp(j) exactly, so the remaining disturbance scales
    as |U|^3.  (The literal uniform 1/6 would leave an O(|U|) error on the
    axis links.)"""
    U = np.array([0.02, -0.015, 0.01])
    e1, m1 = _comoving_error(U)
    e2, m2 = _comoving_error(U / 2)
    assert 7.0 < e1 / e2 < 9.0 and 7.0 < m1 / m2 < 9.0
    e3, m3 = _comoving_error(U / 20)
    assert e3 < 1e-9 and m3 < 2e-9


def _droplet_pressure_jump(radius, g=0.15, L=48, steps=2500):
    """Cylindrical red droplet in blue (nz = 1), started from the flat
    interface's coexisting bulk densities at this g (0.840 / 0.005, found by
    relaxing a flat lamella); returns (p_in - p_out, equimolar radius)."""
    yy, xx = np.mgrid[0:L, 0:L]
    r = np.sqrt((xx - L / 2 + 0.5) ** 2 + (yy - L / 2 + 0.5) ** 2)
    inside = 0.5 * (1.0 - np.tanh((r - radius) / 1.5))
    rho = np.zeros((2, L * L))
    rho[0] = (0.00485 + 0.83474 * inside).reshape(-1)
    rho[1] = (0.00485 + 0.83474 * (1.0 - inside)).reshape(-1)
    o = ref.Oracle(nx=L, ny=L, nz=1, n_particles=0, g_br=g, noise_amp=0.0)
    o.init_fields(rho)
    o.step(steps)
    rr = o.rho()
    psi = 1.0 - np.exp(-rr)  # Eq. eqn_ref_dens with rho0 = 1
    # bulk pressure of the two-component Shan-Chen fluid: the force of Eq.
    # eqn_shan-chen-F is -g A grad(Psi^r Psi^b) to leading order, A =
    # sum_i W_i c_ix^2 = 2 * 2 + 8 * 1 = 12 for the (2, 1) weights
    p = (CS2 * (rr[0] + rr[1]) + g * 12.0 * psi[0] * psi[1]).reshape(L, L)
    c = L // 2
    p_in = p[c - 2:c + 2, c - 2:c + 2].mean()
    p_out = p[0:3, 0:3].mean()
    red = rr[0].reshape(L, L)
    area = np.sum((red - red[0, 0]) / (red[c, c] - red[0, 0]))
    return p_in - p_out, np.sqrt(area / np.pi)


def test_laplace_law_static_droplet():
    """Laplace law for a static droplet (the theory behind the interfaces of
    Secs. II and V): in two dimensions the pressure jump across a circular
    interface is sigma / R with one surface tension sigma for every radius.
    A wrong sign or a dropped factor in the force either dissolves the
    droplet or breaks the 1/R scaling."""
    res = [_droplet_pressure_jump(R0) for R0 in (7.0, 10.0, 14.0)]
    dp = np.array([d for d, _ in res])
    R = np.array([r for _, r in res])
    assert np.all(dp > 0), dp
    sigma = dp * R
    assert np.max(np.abs(sigma / sigma.mean() - 1.0)) < 0.04, sigma
    slope, icpt = np.polyfit(1.0 / R, dp, 1)
    assert abs(icpt) < 0.1 * dp.min(), (slope, icpt)


def test_stokes_drag_periodic_array():
    """Drag on a fixed sphere in a periodic box of side L with the fluid
    driven by a body force (bounce-back and momentum exchange of Eqs.
    eqn_bounce-back and eqn_bounce-back-force): Stokes' 6 pi eta a U times
    Hasimoto's periodic-array factor K(phi) (J. Fluid Mech. 5, 317 (1959);
    the series of Sangani & Acrivos, Int. J. Multiphase Flow 8, 343 (1982)),
    U the mean velocity over the cell and eta = rho c_s^2 (tau - 1/2).  The
    flow starts at about its steady mean velocity so that it settles within
    a few hundred steps.  Bounce-back places the wall within a fraction of a
    node of the input radius; 5 % covers that at R = 4."""
    L, R, gb = 32, 4.0, 1e-6
    P = np.zeros((1, 9))
    P[0, 0:3] = (L / 2 - 0.3, L / 2 + 0.2, L / 2 - 0.1)
    o = ref.Oracle(nx=L, ny=L, nz=L, n_particles=1, radius=R, g_br=0.0, noise_amp=0.0, fixed_particles=1,
                   body_force=(gb, 0.0, 0.0), rho_init=(0.5, 0.5))
    u0 = np.zeros((3, L ** 3))
    u0[0] = 1.7e-3
    o.init_fields(np.full((2, L ** 3), 0.5), u=u0, particles=P)
    o.step(750)
    F, _ = o.particle_forces()
    st = o.get_state()
    fluid = st["owner"] == -1
    c, _, _ = ref.lattice()
    rho = st["f"].sum(axis=(0, 1))
    jx = np.einsum("cin,i->n", st["f"], c[:, 0].astype(np.float64))
    # physical momentum includes half the body force (Sec. II velocity shift)
    U = np.sum(jx[fluid] + 0.5 * rho[fluid] * gb) / 1.0 / L ** 3
    eta = 1.0 * CS2 * (1.0 - 0.5)
    phi = 4.0 / 3.0 * np.pi * R ** 3 / L ** 3
    K = 1.0 / (1 - 1.7601 * phi ** (1 / 3) + phi - 1.5593 * phi ** 2 + 3.9799 * phi ** (8 / 3)
               - 3.0734 * phi ** (10 / 3))
    ratio = F[0, 0] / (6 * np.pi * eta * R * U * K)
    assert abs(ratio - 1.0) < 0.05, ratio
    assert np.all(np.abs(F[0, 1:]) < 1e-3 * F[0, 0]), F


def test_static_sphere_in_fluid_at_rest():
    """No flow appears around a resting sphere in a resting fluid, and the
    bounce-back force on a sphere centred on a node is zero by symmetry."""
    o = ref.Oracle(nx=14, ny=14, nz=14, n_particles=1, radius=3.5, g_br=0.0)
    P = np.zeros((1, 9))
    P[0, 0:3] = (7.0, 7.0, 7.0)
    o.init_fields(np.full((2, 14 ** 3), 0.6), particles=P)
    o.step(5)
    assert np.max(np.abs(o.velocity())) < 1e-15
    F, T = o.particle_forces()
    assert np.max(np.abs(F)) < 1e-12 and np.max(np.abs(T)) < 1e-12


def test_drag_and_torque_oppose_motion():
    """A prescribed translation or rotation of a sphere in fluid at rest is
    resisted: F.U < 0 and T.omega < 0 (Eqs. eqn_bounce-back-force and the
    torque D with r from the centre to the reflection site)."""
    for U, W in (((0.02, 0, 0), (0, 0, 0)), ((0, 0, 0), (0, 0, 0.01)), ((0, 0.01, 0), (0.005, 0, 0))):
        P = np.zeros((1, 9))
        P[0, 0:3] = (8.2, 7.9, 8.4)
        P[0, 3:6] = U
        P[0, 6:9] = W
        o = ref.Oracle(nx=16, ny=16, nz=16, n_particles=1, radius=4.0, g_br=0.0,
                       fixed_particles=1)
        o.init_fields(np.full((2, 16 ** 3), 0.6), particles=P)
        o.step(30)
        F, T = o.particle_forces()
        if np.any(U):
            assert np.dot(F[0], U) < 0
        if np.any(W):
            assert np.dot(T[0], W) < 0


# -------------------------------------------------------- cover / uncover
def test_refill_density_and_momentum():
    """Uncovered nodes are refilled with rho_new^c = mean rho^c over the
    neighbours that were fluid (Eq. eqn_rho_neu) and f = f^eq(rho_new, u_s)
    so that sum_i f = rho_new and sum_i f c = rho_new u_s, u_s = U + w x r;
    covered nodes lose all fluid.  Checked by brute force on the node lists."""
    shape = (14, 13, 12)
    nx, ny, nz = shape
    P = np.zeros((1, 9))
    P[0, 0:3] = (6.3, 6.6, 5.8)
    P[0, 3:6] = (0.3, -0.2, 0.25)   # large, to move across nodes in one MD step
    P[0, 6:9] = (0.02, 0.01, -0.03)
    o = ref.Oracle(nx=nx, ny=ny, nz=nz, n_particles=1, radius=3.4, g_br=0.1,
                   particle_density=50.0)
    o.init_fields(lbinputs.mixture(shape, amp=0.05, seed=21), particles=P)
    o.step(1)                   # moves the particle: X += U
    before = o.get_state()
    rho_b = o.rho()
    o.debug_remap()
    after = o.get_state()
    c, w, _ = ref.lattice()
    X = before["particles"][0, 0:3]
    U = before["particles"][0, 3:6]
    W = before["particles"][0, 6:9]
    L = np.array(shape, float)
    unc = np.nonzero((before["owner"] == 0) & (after["owner"] == -1))[0]
    cov = np.nonzero((before["owner"] == -1) & (after["owner"] == 0))[0]
    assert len(unc) > 0 and len(cov) > 0
    for n in unc:
        x, y, z = n % nx, (n // nx) % ny, n // (nx * ny)
        r = np.array([x, y, z], float) - X
        r -= L * np.round(r / L)
        us = U + np.cross(W, r)
        for comp in range(2):
            vals = []
            for i in range(1, 19):
                m = ((x + c[i, 0]) % nx) + nx * (((y + c[i, 1]) % ny) + ny * ((z + c[i, 2]) % nz))
                if before["owner"][m] == -1:
                    vals.append(rho_b[comp, m])
            f = after["f"][comp, :, n]
            assert abs(f.sum() - np.mean(vals)) < 1e-14
            assert np.allclose(f @ c, np.mean(vals) * us, atol=1e-14)
    for n in cov:
        assert np.all(after["f"][:, :, n] == 0.0)


def test_mass_correction_direction():
    """Eq. masscorr: when the fluid has gained mass the refill is scaled
    down, when it has lost mass scaled up, linearly in C0."""
    shape = (14, 13, 12)
    P = np.zeros((1, 9))
    P[0, 0:3] = (6.3, 6.6, 5.8)
    P[0, 3:6] = (0.3, -0.2, 0.25)
    res = {}
    for c0, dm in ((0.0, 0.0), (20.0, +0.05), (20.0, -0.05), (40.0, -0.05)):
        o = ref.Oracle(nx=14, ny=13, nz=12, n_particles=1, radius=3.4, g_br=0.1,
                       particle_density=50.0, mass_corr_c0=c0)
        o.init_fields(lbinputs.mixture(shape, amp=0.05, seed=21), particles=P)
        o.step(1)
        st = o.get_state()
        mass = o.observe()["mass"]
        st["meta"][1] = mass[0] - dm * 14 * 13 * 12   # pretend the initial mass differed
        st["meta"][2] = mass[1] - dm * 14 * 13 * 12
        o.set_state(st)
        unc_before = st["owner"] == 0
        o.debug_remap()
        after = o.get_state()
        unc = np.nonzero(unc_before & (after["owner"] == -1))[0]
        res[(c0, dm)] = after["f"][0][:, unc].sum(axis=0)
    base = res[(0.0, 0.0)]
    up = res[(20.0, +0.05)] / base
    down = res[(20.0, -0.05)] / base
    down2 = res[(40.0, -0.05)] / base
    assert np.all(up < 1.0) and np.all(down > 1.0)
    assert np.allclose(down2 - 1.0, 2 * (down - 1.0), rtol=1e-12)


def masscorr_factors():
    """Refill densities of the uncovered nodes of one remap with a planted
    total mass error Delta M^c per component, divided by the same refill
    without the correction: (measured factors, expected factors) per
    component.  Expected, from Eq. masscorr with N the number of all lattice
    sites (fluid and solid) and unequal initial densities so that the ratio
    sum_c' rho_init^c' / rho_init^c differs between the components:
    1 - C0 (0.42 + 0.28) / rho_init^c Delta M^c / N."""
    nx, ny, nz = 14, 13, 12
    N = nx * ny * nz
    rho_init = (0.42, 0.28)
    dM = (0.9, -1.3)          # planted mass errors (current minus initial)
    c0 = 3.0
    P = np.zeros((1, 9))
    P[0, 0:3] = (6.3, 6.6, 5.8)
    P[0, 3:6] = (0.3, -0.2, 0.25)
    rho = lbinputs.mixture((nx, ny, nz), rho_init=rho_init, amp=0.02, seed=23)
    got = {}
    for corr in (0.0, c0):
        o = ref.Oracle(nx=nx, ny=ny, nz=nz, n_particles=1, radius=3.4, g_br=0.1, rho_init=rho_init,
                       particle_density=50.0, mass_corr_c0=corr)
        o.init_fields(rho, particles=P)
        o.step(1)
        st = o.get_state()
        mass = o.observe()["mass"]
        st["meta"][1] = mass[0] - dM[0]
        st["meta"][2] = mass[1] - dM[1]
        o.set_state(st)
        unc_before = st["owner"] == 0
        o.debug_remap()
        after = o.get_state()
        unc = np.nonzero(unc_before & (after["owner"] == -1))[0]
        assert len(unc) > 0
        got[corr] = np.stack([after["f"][c][:, unc].sum(axis=0) for c in range(2)])
    measured = got[c0] / got[0.0]
    expected = [1.0 - c0 * (0.42 + 0.28) / rho_init[c] * dM[c] / N for c in range(2)]
    return measured, expected


def test_mass_correction_magnitude():
    """Eq. masscorr, magnitude: the refill of every uncovered node is scaled
    by 1 - C0 (sum_c' rho_init^c' / rho_init^c) Delta M^c / N with N the
    total number of lattice sites (Sec. IV names it so), per component.  A
    fluid-node count in place of N, a swapped density ratio or a dropped
    factor changes the factor by far more than rounding."""
    measured, expected = masscorr_factors()
    for c in range(2):
        assert np.allclose(measured[c], expected[c], rtol=0, atol=1e-13), (c, measured[c][:4], expected[c])


def lubrication_cases():
    """(measured, expected) normal lubrication forces on particle p.

    Expected from the leading-order Reynolds lubrication force between two
    spheres of radii a1, a2 approaching at normal speed v with surface gap h
    (e.g. Kim & Karrila, Microhydrodynamics, Ch. 9):
        F = 6 pi eta (a1 a2 / (a1 + a2))^2 v / h,
    repulsive; Eq. eqn_ladd_lubrikation adds only the part the lattice does
    not resolve, 1/h - 1/h_c, with the gap clamped at h_min, and the LB
    viscosity eta = rho0 c_s^2 (tau - 1/2) (rho0 = 1) at the mean tau of the
    two components."""
    out = []
    hc, hmin = 2.0 / 3.0, 0.1
    for R, tau, gap, v in ((5.0, (0.8, 1.4), 0.3, 0.01), (5.0, (0.8, 1.4), 0.05, 0.01),
                           (3.0, (1.0, 1.0), 0.45, 0.02), (7.5, (0.6, 0.9), 0.2, 0.004)):
        eta = CS2 * (0.5 * (tau[0] + tau[1]) - 0.5)
        a_red = R * R / (R + R)
        h = max(gap, hmin)
        want = 6.0 * np.pi * eta * a_red ** 2 * v * (1.0 / h - 1.0 / hc)
        # p on +x of q, moving towards it at speed v
        Fp = ref.pair_force((2 * R + gap, 0, 0), (0, 0, 0), (-v, 0, 0), (0, 0, 0), nx=64, ny=64, nz=64,
                            radius=R, tau=tau, k_hertz=0.0, lub_cut=hc, lub_min=hmin)
        out.append((Fp[0], want))
    return out


def test_lubrication_magnitude():
    """Eq. eqn_ladd_lubrikation, magnitude: the oracle's force equals the
    Reynolds lubrication force of two equal spheres (reduced radius R / 2)
    above the cut-off correction, at four radii / viscosities / gaps, one of
    them clamped.  A 3 pi for 6 pi, R^2 for R^4 / (2R)^2 or a single
    component's tau in the viscosity fails it."""
    for got, want in lubrication_cases():
        assert want > 0.0
        assert abs(got - want) < 1e-12 * want, (got, want)


# ------------------------------------------------------ colour and symmetry
def _interface_particle(color, swap=False):
    n = 16
    rho = lbinputs.lamellae((n, n, n), axis=2, rho_major=0.7, rho_minor=0.05)
    if swap:
        rho = rho[::-1].copy()
    P = np.zeros((1, 9))
    P[0, 0:3] = (7.5, 7.5, n / 2 - 0.5)
    o = ref.Oracle(nx=n, ny=n, nz=n, n_particles=1, radius=3.5, g_br=0.2, color=color,
                   fixed_particles=1)
    o.init_fields(rho, particles=P)
    o.step(1)
    return o.particle_forces()[0][0]


def test_colour_sign_and_red_blue_symmetry():
    """Sec. IV: positive colour adds red virtual fluid, which pulls the
    particle into the red phase (here z < n/2); negative colour into the
    blue.  With zero colour the mirror-symmetric set-up gives no normal
    force (theta = 90 deg).  Swapping red and blue together with the sign of
    the colour mirrors the force."""
    f0 = _interface_particle(0.0)
    assert abs(f0[2]) < 1e-13
    fp = _interface_particle(+0.05)
    fm = _interface_particle(-0.05)
    assert fp[2] < -1e-6 and fm[2] > 1e-6
    fsw = _interface_particle(-0.05, swap=True)
    assert abs(fsw[2] - fp[2]) < 1e-12 * max(1.0, abs(fp[2])) + 1e-14


def test_virtual_fluid_removes_density_halo():
    """Fig. 1: with the shell filled by virtual fluid the total density next
    to a particle stays at the bulk value; with an empty particle (the
    original algorithm) a layer of increased density forms."""
    n = 20
    P = np.zeros((1, 9))
    P[0, 0:3] = (10.0, 10.0, 10.0)
    out = {}
    for vf in (1, 0):
        o = ref.Oracle(nx=n, ny=n, nz=n, n_particles=1, radius=4.0, g_br=0.08,
                       virtual_fluid=vf, fixed_particles=1)
        o.init_fields(np.full((2, n ** 3), 0.35), particles=P)
        o.step(300)
        r = o.rho().sum(axis=0).reshape(n, n, n)
        owner = o.get_state()["owner"].reshape(n, n, n)
        zz, yy, xx = np.indices((n, n, n))
        d = np.sqrt((xx - 10.0) ** 2 + (yy - 10.0) ** 2 + (zz - 10.0) ** 2)
        near = (owner == -1) & (d < 5.5)
        far = (owner == -1) & (d > 8.5)
        out[vf] = r[near].mean() / r[far].mean() - 1.0
    assert abs(out[1]) < 0.005
    assert out[0] > 3 * abs(out[1]) and out[0] > 0.005


# ---------------------------------------------------------------- MD forces
def test_hertz_force_is_minus_gradient():
    """Eq. eq:hertz: the contact force is -dV/dr of V = K (2R - r)^{5/2}."""
    R, K = 5.0, 1.7
    for d in (9.2, 9.7, 9.95):
        Fp = ref.pair_force((d, 0, 0), (0, 0, 0), (0, 0, 0), (0, 0, 0), nx=64, ny=64, nz=64,
                            radius=R, k_hertz=K, lub_cut=-1.0)
        V = lambda r: K * (2 * R - r) ** 2.5
        h = 1e-6
        dVdr = (V(d + h) - V(d - h)) / (2 * h)
        assert abs(Fp[0] - (-dVdr)) < 1e-6 * abs(dVdr)
        assert Fp[1] == 0 and Fp[2] == 0
    assert np.all(ref.pair_force((10.01, 0, 0), (0, 0, 0), (0, 0, 0), (0, 0, 0), nx=64, ny=64, nz=64,
                                 radius=R, lub_cut=-1.0) == 0)


def test_lubrication_properties():
    """Eq. eqn_ladd_lubrikation: acts only below the cut-off gap, vanishes
    continuously there, is clamped below h_min, opposes the relative normal
    velocity, and is linear in it; the minimum image is used across the
    periodic boundary."""
    R = 5.0
    kw = dict(nx=64, ny=64, nz=64, radius=R, k_hertz=0.0)
    approach = ((0, 0, 0), (-0.01, 0, 0))   # p at +x moves toward q
    f = lambda d, U=approach: ref.pair_force((d, 0, 0), (0, 0, 0), U[1], U[0], **kw)[0]
    assert f(10.0 + 0.7) == 0.0
    assert abs(f(10.0 + 2.0 / 3.0 - 1e-9)) < 1e-9
    assert f(10.3) > 0                       # repulsive when approaching
    assert f(10.05) == f(10.1) == f(10.0)    # clamped at h_min
    assert abs(f(10.3, ((0, 0, 0), (-0.02, 0, 0))) - 2 * f(10.3)) < 1e-15
    sep = ((0, 0, 0), (0.01, 0, 0))
    assert f(10.3, sep) == -f(10.3)
    tang = ((0, 0, 0), (0, 0.01, 0))
    assert f(10.3, tang) == 0.0
    # across the periodic boundary: p at x = 63, q at x = 9.7 -> gap 0.7 - 1 = ...
    Fw = ref.pair_force((63.0, 0, 0), (9.2, 0, 0), (0.01, 0, 0), (0, 0, 0), **kw)
    assert Fw[0] < 0                          # p sits at -1 relative to q, approaching: pushed to -x


# ------------------------------------------------------------ seeded init
def test_seeded_init_placement_and_noise():
    """Random sequential addition gives non-overlapping spheres (minimum
    image distance >= 2R) with the count from the volume fraction, and node
    densities within rho_init +- a."""
    o = ref.Oracle(nx=32, ny=32, nz=32, n_particles=-1, volume_fraction=0.13, radius=4.0,
                   noise_amp=0.01)
    assert o.np == int(np.floor(0.13 * 32 ** 3 / (4 / 3 * np.pi * 64) + 0.5))
    o.init_from_seed(7)
    st = o.get_state()
    X = st["particles"][:, 0:3]
    L = 32.0
    for a, b in itertools.combinations(range(o.np), 2):
        d = X[a] - X[b]
        d -= L * np.round(d / L)
        assert np.dot(d, d) >= 64.0 - 1e-12
    r = o.rho()
    fl = st["owner"] == -1
    assert np.all(np.abs(r[:, fl] - 0.7) <= 0.01 + 1e-15)
    assert abs(r[:, fl].mean() - 0.7) < 1e-3
    # every node within R of a centre is solid, every other node is fluid
    zz, yy, xx = np.indices((32, 32, 32))
    pos = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], 1).astype(float)
    inside = np.zeros(32 ** 3, bool)
    for q in range(o.np):
        d = pos - X[q]
        d -= L * np.round(d / L)
        inside |= (d ** 2).sum(1) <= 16.0
    assert np.array_equal(inside, st["owner"] >= 0)


# --------------------------------------------------------------- analysis
def test_domain_size_of_sine_pattern():
    """Eq. eq:domsize on single and mixed Fourier modes.  A product of sines
    has all its power at |k_i| = 2 pi / lam_i, so L_i = lam_i; a sum of three
    sines of equal amplitude puts a third of the power on each axis, so
    <k_x^2> = (2 pi / lam_x)^2 / 3 and L_x = lam_x sqrt(3)."""
    n = 32
    z, y, x = np.indices((n, n, 24))
    phi1 = np.sin(2 * np.pi * x / 8.0) * np.sin(2 * np.pi * y / 16.0) * np.sin(2 * np.pi * z / 32.0)
    assert np.allclose(oan.domain_size(phi1), (8.0, 16.0, 32.0), atol=1e-9)
    phi = np.sin(2 * np.pi * x / 8.0) + np.sin(2 * np.pi * y / 16.0) + np.sin(2 * np.pi * z / 32.0)
    assert np.allclose(oan.domain_size(phi), np.sqrt(3.0) * np.array([8.0, 16.0, 32.0]), atol=1e-9)


def test_interface_height_and_angle():
    """Eq. eqn_contactangle_calculation with the interface at the linearly
    interpolated zero of phi."""
    col = np.array([1.0, 0.6, 0.2, -0.2, -0.6])
    assert abs(oan.interface_height(col) - 2.5) < 1e-15
    assert abs(oan.contact_angle(-2.93, 10.0) - 107.04) < 0.01
    assert oan.contact_angle(0.0, 5.0) == 90.0


def test_coverage_brute_force():
    """Interface coverage (a reading: the paper does not define it), checked
    against a per-node loop on a hand-built 7^3 box: particle 0 touches both
    phases, particle 1 only phi > 0, particle 2 only fluid at phi = 0 (counts
    as neither side)."""
    n = 7
    owner = -np.ones((n, n, n), np.int32)
    phi = np.ones((n, n, n))
    owner[1, 1, 1] = 0
    phi[1, 1, 2] = -0.5          # a diagonal-free axis neighbour of particle 0
    owner[5, 5, 5] = 1           # surrounded by phi = 1 only
    owner[3, 5, 1] = 2
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if 0 < abs(dx) + abs(dy) + abs(dz) <= 2:
                    phi[(3 + dz) % n, (5 + dy) % n, (1 + dx) % n] = 0.0
    # brute force over the D3Q19 neighbours of every solid node
    signs = {0: set(), 1: set(), 2: set()}
    for z in range(n):
        for y in range(n):
            for x in range(n):
                p = owner[z, y, x]
                if p < 0:
                    continue
                for dz in (-1, 0, 1):
                    for dy in (-1, 0, 1):
                        for dx in (-1, 0, 1):
                            if not 0 < abs(dx) + abs(dy) + abs(dz) <= 2:
                                continue
                            q = ((z + dz) % n, (y + dy) % n, (x + dx) % n)
                            if owner[q] == -1 and phi[q] != 0:
                                signs[p].add(np.sign(phi[q]))
    expect = np.mean([len(signs[p]) == 2 for p in range(3)])
    assert expect == 1.0 / 3.0
    assert oan.coverage(phi, owner, 3) == expect
    # a node two links away (x + 2) is not a neighbour
    phi2 = phi.copy()
    phi2[1, 1, 2] = 1.0
    phi2[1, 1, 3] = -1.0
    assert oan.coverage(phi2, owner, 3) == 0.0


# ------------------------------------------------------------- spheroids
SPH = dict(radius=4.0, aspect=1.75)  # semi-axes 4, 4, 7


def _unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v)


def test_spheroid_inside_test_and_volume():
    """Spheroid with semi-axes R, R, c about e (the generality the paper
    claims for the coupling, Secs. I and III): the oracle's inside test
    equals (d.e)^2 / c^2 + |d x e|^2 / R^2 <= 1 away from the boundary, and
    the lattice nodes it counts approach 4/3 pi R^2 c."""
    rng = np.random.default_rng(5)
    R, c = SPH["radius"], SPH["radius"] * SPH["aspect"]
    for _ in range(2000):
        e = _unit(rng.normal(size=3))
        d = rng.uniform(-8, 8, size=3)
        q = np.dot(d, e) ** 2 / c ** 2 + np.sum(np.cross(d, e) ** 2) / R ** 2
        if abs(q - 1.0) < 1e-9:
            continue
        assert ref.inside(d, e, **SPH) == (q <= 1.0)
    e = _unit([0.3, -0.5, 0.8])
    X = np.array([0.37, 0.21, 0.64])
    g = np.arange(-9, 10)
    D = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) - X
    n = sum(ref.inside(d, e, **SPH) for d in D)
    assert abs(n / (4.0 / 3.0 * np.pi * R * R * c) - 1.0) < 0.03, n


def test_spheroid_claims_and_placement():
    """Seeded spheroids: each solid node lies inside its owner (the inside
    test with the particle's own axis), axes are unit vectors, and the node
    count per particle is near the volume."""
    o = ref.Oracle(nx=40, ny=40, nz=40, n_particles=6, g_br=0.0, **SPH)
    o.init_from_seed(7)
    st = o.get_state()
    E = o.axes()
    assert np.allclose(np.linalg.norm(E, axis=1), 1.0)
    assert not np.allclose(E, [0, 0, 1])
    z, y, x = np.unravel_index(np.arange(40 ** 3), (40, 40, 40))
    own = st["owner"]
    R, c = SPH["radius"], SPH["radius"] * SPH["aspect"]
    for q in range(6):
        sel = np.nonzero(own == q)[0]
        Xq = st["particles"][q, :3]
        d = np.stack([x[sel], y[sel], z[sel]], 1) - Xq
        d -= 40 * np.round(d / 40)
        assert all(ref.inside(v, E[q], **SPH) for v in d[::7])
        assert abs(len(sel) / (4.0 / 3.0 * np.pi * R * R * c) - 1.0) < 0.05


def test_spheroid_contact_distance():
    """Contact distance along the line of centres: 2R for spheres, 2c end to
    end, 2R side by side, R + c for a T configuration."""
    R, c = SPH["radius"], SPH["radius"] * SPH["aspect"]
    ez, ex = np.array([0, 0, 1.0]), np.array([1.0, 0, 0])
    assert ref.contact_distance(ez, ex, ex, radius=R) == 2 * R
    assert abs(ref.contact_distance(ez, ez, ez, **SPH) - 2 * c) < 1e-12
    assert abs(ref.contact_distance(ez, ex, ex, **SPH) - 2 * R) < 1e-12
    assert abs(ref.contact_distance(ez, ez, ex, **SPH) - (R + c)) < 1e-12


def test_free_rotation_of_a_spheroid():
    """Torque-free rotation (Euler's equations of a symmetric top): spin
    about the symmetry axis leaves e fixed; spin perpendicular to it turns e
    by |omega| per step in that plane; in general L = I(e) omega is
    conserved and e precesses about L at |L| / I_perp while keeping its
    angle to L (exactly, for the update that turns e about L).  A swapped
    I_par / I_perp or a wrong inverse fails this."""
    m = SPH.get("particle_density", 1.0) * 4.0 / 3.0 * np.pi * SPH["radius"] ** 2 * SPH["radius"] * SPH["aspect"]
    R, c = SPH["radius"], SPH["radius"] * SPH["aspect"]
    Ipar, Iperp = 0.4 * m * R * R, 0.2 * m * (R * R + c * c)
    T0 = np.zeros(3)
    e0 = _unit([0.2, -0.3, 0.9])
    W, e = ref.rotate(0.01 * e0, e0, T0, **SPH)
    assert np.allclose(e, e0, atol=1e-15) and np.allclose(W, 0.01 * e0, atol=1e-15)
    w = 0.003
    W, e = np.array([0.0, w, 0.0]), np.array([0.0, 0.0, 1.0])
    for _ in range(100):
        W, e = ref.rotate(W, e, T0, **SPH)
    assert np.allclose(e, [np.sin(100 * w), 0.0, np.cos(100 * w)], atol=1e-12)
    e = _unit([0.1, 0.2, 0.97])
    W = np.array([0.004, -0.002, 0.006])

    def Lof(W, e):
        return Iperp * W + (Ipar - Iperp) * np.dot(e, W) * e

    L0 = Lof(W, e)
    Lh = L0 / np.linalg.norm(L0)
    cos0 = np.dot(e, Lh)
    e_perp0 = _unit(e - cos0 * Lh)
    n = 400
    for _ in range(n):
        W, e = ref.rotate(W, e, T0, **SPH)
    assert np.allclose(Lof(W, e), L0, rtol=1e-12, atol=1e-16)
    assert abs(np.dot(e, Lh) - cos0) < 1e-12
    ep = _unit(e - np.dot(e, Lh) * Lh)
    ang = np.arctan2(np.dot(np.cross(e_perp0, ep), Lh), np.dot(e_perp0, ep))
    expect = np.mod(n * np.linalg.norm(L0) / Iperp + np.pi, 2 * np.pi) - np.pi
    assert abs(ang - expect) < 1e-9, (ang, expect)


def test_spheroid_momentum_conserved_in_fluid():
    """Moving, rotating spheroids exchange momentum with the fluid through
    the same links, cover/uncover and contact forces as spheres: fluid plus
    particle momentum is conserved to rounding."""
    o = ref.Oracle(nx=28, ny=24, nz=30, n_particles=3, g_br=0.1, color=0.02, particle_density=3.0, **SPH)
    o.init_from_seed(11)
    st = o.get_state()
    P = st["particles"].copy()
    P[:, 3:6] = [[0.05, -0.03, 0.02], [-0.04, 0.02, 0.03], [0.01, 0.05, -0.04]]
    P[:, 6:9] = [[0.01, 0.02, -0.01], [0.0, -0.02, 0.015], [0.02, 0.0, 0.01]]
    E = o.axes()
    o2 = ref.Oracle(nx=28, ny=24, nz=30, n_particles=3, g_br=0.1, color=0.02, particle_density=3.0, **SPH)
    o2.set_axes(E)
    o2.init_fields(lbinputs.mixture((28, 24, 30), amp=0.05, seed=12), particles=P)
    ob0 = o2.observe()
    p0 = ob0["mom_fluid"] + ob0["mom_part"]
    o2.step(30)
    ob = o2.observe()
    assert ob["n_cover"] > 0 and ob["n_uncover"] > 0
    p1 = ob["mom_fluid"] + ob["mom_part"]
    assert np.all(np.abs(p1 - p0) < 1e-12 * (ob["mass"].sum() + 1)), p1 - p0
    assert not np.allclose(o2.axes(), E)


def test_overlapping_spheroids_claims_brute_force():
    """Two overlapping spheroids (reading #12 with the spheroid inside test):
    a node inside either is solid, and a node inside both goes to the nearer
    centre (the lower index on a tie); checked against a brute-force loop."""
    L = 24
    P = np.zeros((2, 9))
    P[0, :3] = (10.3, 11.6, 12.2)
    P[1, :3] = (14.1, 12.4, 11.7)
    E = np.array([_unit([1.0, 0.2, 0.1]), _unit([-0.3, 1.0, 0.4])])
    o = ref.Oracle(nx=L, ny=L, nz=L, n_particles=2, g_br=0.0, fixed_particles=1, **SPH)
    o.set_axes(E)
    o.init_fields(np.full((2, L ** 3), 0.5), particles=P)
    own = o.get_state()["owner"].reshape(L, L, L)
    both = 0
    for z in range(L):
        for y in range(L):
            for x in range(L):
                best, bd = -1, None
                for q in range(2):
                    d = np.array([x, y, z], float) - P[q, :3]
                    d -= L * np.round(d / L)
                    if ref.inside(d, E[q], **SPH):
                        d2 = float(np.dot(d, d))
                        if best >= 0:
                            both += 1
                        if bd is None or d2 < bd:
                            best, bd = q, d2
                assert own[z, y, x] == best, (x, y, z, own[z, y, x], best)
    assert both > 20


# ------------------------------------- implicit particle update (reading #18)
def _link_drag(o, X, rho_tot):
    """Z = sum over the links of the particle of 6 zeta_j rho a a^T with
    a = (c_j, r x c_j), r from the centre X to the link midpoint: the
    derivative of the links' force and torque with respect to (U, omega)
    under Eq. eqn_ladd_bewegtewand, written out from the geometry."""
    c, w, _ = ref.lattice()
    c = c.astype(np.float64)
    nx, ny, nz = o.nx, o.ny, o.nz
    owner = o.get_state()["owner"].reshape(nz, ny, nx)
    L = np.array([nx, ny, nz], np.float64)
    Z = np.zeros((6, 6))
    zz, yy, xx = np.nonzero(owner == -1)
    pos = np.stack([xx, yy, zz], axis=1).astype(np.float64)
    for j in range(1, 19):
        t = (pos + c[j]).astype(int) % np.array([nx, ny, nz])
        hit = owner[t[:, 2], t[:, 1], t[:, 0]] == 0
        r = pos[hit] + 0.5 * c[j] - X
        r -= L * np.round(r / L)
        a = np.concatenate([np.broadcast_to(c[j], r.shape), np.cross(r, c[j])], axis=1)
        Z += 6.0 * w[j] * rho_tot * a.T @ a
    return Z


@pytest.mark.parametrize("implicit", [0, 1])
def test_first_step_velocity_of_a_sphere_in_fluid_at_rest(implicit):
    """A sphere centred on a node of a uniform fluid at rest (g = 0, tau = 1):
    by the cubic symmetry of its links the populations' part of the link
    force and torque cancels, so the only force is the wall term's -Z V0.
    Explicit update (reading #8): V1 = V0 - M^-1 Z V0.  Implicit update
    (reading #18): (M + Z)(V1 - V0) = -Z V0, i.e. V1 = (M + Z)^-1 M V0.
    Z comes from the link geometry (_link_drag); a light sphere (rho_p = 0.5)
    makes the two results differ at first order."""
    n, R, rhop, rho_c = 16, 3.5, 0.5, 0.35
    o = ref.Oracle(nx=n, ny=n, nz=n, n_particles=1, radius=R, g_br=0.0, particle_density=rhop,
                   rho_init=(rho_c, rho_c), implicit_update=implicit)
    V0 = np.array([0.01, -0.005, 0.003, 0.001, 0.002, -0.0015])
    P = np.zeros((1, 9))
    P[0, 0:3] = 8.0
    P[0, 3:9] = V0
    o.init_fields(np.full((2, n ** 3), rho_c), particles=P)
    Z = _link_drag(o, P[0, 0:3], 2 * rho_c)
    m = rhop * 4.0 / 3.0 * np.pi * R ** 3
    M = np.diag([m, m, m, 0.4 * m * R * R, 0.4 * m * R * R, 0.4 * m * R * R])
    o.step(1)
    V1 = o.get_state()["particles"][0, 3:9]
    want = np.linalg.solve(M + Z, M @ V0) if implicit else V0 - np.linalg.solve(M, Z @ V0)
    assert np.max(np.abs(Z @ V0)) > 0.05 * np.max(np.abs(M @ V0))  # the wall term matters here
    assert np.max(np.abs(V1 - want)) < 1e-13, (V1, want)


@pytest.mark.parametrize("rhop", [1.0, 3.0])
def test_implicit_update_conserves_momentum(rhop):
    """With the implicit update each link's bounce-back population also gets
    the wall term of the velocity change, so fluid plus particle momentum
    stays exact, as in the explicit case above (moving, colliding, covering
    and uncovering spheres, colours, mass correction)."""
    shape = (20, 18, 16)
    P = lbinputs.spheres(shape, 3.2, 4, seed=11, min_gap=0.3, vmax=0.04, wmax=0.02)
    o = ref.Oracle(nx=20, ny=18, nz=16, n_particles=4, radius=3.2, g_br=0.15, color=0.04,
                   particle_density=rhop, mass_corr_c0=5.0, implicit_update=1)
    o.set_colors(np.array([0.04, -0.03, 0.0, 0.05]))
    o.init_fields(lbinputs.mixture(shape, amp=0.05, seed=12), particles=P)
    p0 = _total_momentum(o)
    scale = o.observe()["mass"].sum() * 0.04
    o.step(60)
    ob = o.observe()
    assert ob["n_cover"] > 0 and ob["n_uncover"] > 0
    assert np.all(np.abs(_total_momentum(o) - p0) < 1e-11 * scale)


def test_implicit_update_is_for_spheres_only():
    with pytest.raises(ValueError):
        ref.Oracle(nx=8, ny=8, nz=8, n_particles=0, aspect=1.5, implicit_update=1)
