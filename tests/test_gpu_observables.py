"""Observables computed by the library (lb_observables, lb_export_phi)
against the oracle's analysis of the same exported state.

The domain size of Sec. VI (Eq. eq:domsize) and the interface coverage are
computed on the device (an FP64 FFT per lattice line and axis); the oracle
(oracle/analysis.py) applies numpy's three-dimensional FFT to phi formed on
the host from the exported populations.  Both are FP64: they agree to
1e-10 relative.
"""
import numpy as np
import pytest

import lbinputs
from oracle import analysis as oan

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1004_4414_gb300 import build

    build.build()


def host_phi(st, shape):
    """phi = rho^r - rho^b from the exported populations, 0 on solid nodes."""
    nx, ny, nz = shape
    rho = st["f"].sum(axis=1)
    phi = np.where(st["owner"] == -1, rho[0] - rho[1], 0.0)
    return phi.reshape(nz, ny, nx)


def check_against_oracle(s, shape, np_, box=0):
    st = s.export_state(box)
    phi_h = host_phi(st, shape)
    ob = s.observables(box)
    phi_d = s.phi(box)
    assert np.max(np.abs(phi_d - phi_h)) < 1e-14
    L_o = np.array(oan.domain_size(phi_h))
    assert np.all(np.isfinite(ob["L"]))
    assert np.allclose(ob["L"], L_o, rtol=1e-10, atol=0), (ob["L"], L_o)
    cov_o = oan.coverage(phi_d, st["owner"].reshape(phi_h.shape), np_)
    assert ob["coverage"] == cov_o
    L2, cov2 = s.structure(box)
    assert np.array_equal(L2, ob["L"]) and cov2 == ob["coverage"]
    return ob["L"], ob["coverage"]


def lamella_with_particles(shape, z_interface, inside_red, at_interface, radius=3.0, seed=3):
    """Red below z_interface, blue above (noise on both), spheres: some deep
    in the red layer, some deep in the blue one, some on the interface."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    zz = np.indices((nz, ny, nx))[0].reshape(-1)
    red = zz < z_interface
    rho = np.empty((2, nx * ny * nz))
    rho[0] = np.where(red, 0.65, 0.05) + 0.01 * rng.random(rho.shape[1])
    rho[1] = np.where(red, 0.05, 0.65) + 0.01 * rng.random(rho.shape[1])
    P = []
    for k, z in enumerate([z_interface / 2] * inside_red + [z_interface + (nz - z_interface) / 2] * at_interface):
        P.append([4.5 + 8.0 * k % (nx - 4), 6.0 + 7.0 * k % (ny - 6), z, 0, 0, 0, 0, 0, 0])
    for k in range(at_interface):
        P.append([5.0 + 9.0 * k % (nx - 5), 16.0 + 5.0 * k % (ny - 8), z_interface - 0.3, 0, 0, 0, 0, 0, 0])
    return rho, np.array(P, float)


@pytest.mark.parametrize("shape", [(32, 32, 32), (36, 30, 28), (37, 29, 23)])
def test_domain_size_and_coverage_fp64(shape):
    """A red and a blue layer with spheres inside each layer and on the
    interface: coverage strictly between 0 and 1, and the domain sizes of a
    layered field, on power-of-two and mixed-radix (2 3 5, 37, 29, 23) axes."""
    from paper_1004_4414_gb300 import Simulation

    nx, ny, nz = shape
    rho, P = lamella_with_particles(shape, nz // 2, inside_red=2, at_interface=2)
    np_ = len(P)
    s = Simulation(dict(nx=nx, ny=ny, nz=nz, n_particles=np_, radius=3.0, g_br=0.12, precision="fp64",
                        fixed_particles=1))
    s.init_fields(0, rho, particles=P)
    for steps in (0, 5):
        s.step(steps)
        L, cov = check_against_oracle(s, shape, np_)
        assert 0.0 < cov < 1.0
    s.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_domain_size_seeded_moving_particles(prec):
    """Seeded noise with moving spheres, FP32 and BF16 storage: the library's
    L and coverage equal the oracle analysis of the exported state."""
    from paper_1004_4414_gb300 import Simulation

    shape = (48, 40, 32)
    nx, ny, nz = shape
    s = Simulation(dict(nx=nx, ny=ny, nz=nz, n_particles=10, radius=3.5, g_br=0.2, precision=prec,
                        particle_density=2.0, noise_amp=0.05, rho_init=(0.35, 0.35)))
    s.init_from_seed(5)
    s.step(30)
    check_against_oracle(s, shape, 10)
    s.close()


def test_domain_size_long_lines():
    """A box with an axis longer than 2048 nodes (the FFT of those lines runs
    in global scratch) and a sine pattern along it: L along that axis is the
    wavelength (a single Fourier mode), the oracle agrees."""
    from paper_1004_4414_gb300 import Simulation

    shape = (6, 2100, 4)
    nx, ny, nz = shape
    y = np.indices((nz, ny, nx))[1].reshape(-1)
    lam = 2100 / 15.0
    rho = np.stack([0.35 + 0.1 * np.sin(2 * np.pi * y / lam), 0.35 - 0.1 * np.sin(2 * np.pi * y / lam)])
    s = Simulation(dict(nx=nx, ny=ny, nz=nz, n_particles=0, g_br=0.0, precision="fp64"))
    s.init_fields(0, rho)
    ob = s.observables()
    st = s.export_state()
    L_o = np.array(oan.domain_size(host_phi(st, shape)))
    assert abs(ob["L"][1] - lam) < 1e-9 * lam
    assert np.allclose(ob["L"][1], L_o[1], rtol=1e-10)
    # phi is uniform along x and z: no power there
    assert np.isnan(ob["L"][0]) or ob["L"][0] > 1e6
    s.close()


def test_uniform_phi_gives_nan_domain_size():
    from paper_1004_4414_gb300 import Simulation

    s = Simulation(dict(nx=16, ny=12, nz=10, n_particles=0, g_br=0.0, precision="fp64"))
    s.init_fields(0, np.full((2, 16 * 12 * 10), 0.4))
    ob = s.observables()
    assert np.all(np.isnan(ob["L"])) and ob["coverage"] == 0.0
    s.close()
