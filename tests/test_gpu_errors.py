"""The sticky device error word, provoked from the host.

The kernels check for an unstable state (a non-finite or non-positive
density, |u| >= 0.5 of the node velocity, a particle faster than one node
per step) and for overflowing fixed-capacity lists (the 32-entry neighbour
list, the event list, the shell lists).  They only set a bit and carry on;
no check traps, faults or waits.  Each test builds such a state through the
C ABI and expects lb_sync / lb_step / lb_observables to report the code.
"""
import math

import numpy as np
import pytest

import lbinputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1004_4414_gb300 import build

    build.build()


def expect_error(s, code):
    from paper_1004_4414_gb300.binding import LbError

    with pytest.raises(LbError) as e:
        s.sync()
    assert e.value.code == code
    assert s.observables()["error"] == code
    # sticky: the next call reports it again
    with pytest.raises(LbError) as e2:
        s.step(1)
        s.sync()
    assert e2.value.code == code


@pytest.mark.parametrize("prec", ["fp32", "fp16", "fp64"])
def test_nan_population_reports_unstable(prec):
    from paper_1004_4414_gb300 import Simulation
    from paper_1004_4414_gb300.binding import LB_EUNSTABLE

    s = Simulation(dict(nx=20, ny=16, nz=12, n_particles=0, g_br=0.1, precision=prec))
    s.init_fields(0, lbinputs.mixture((20, 16, 12), amp=0.02, seed=1))
    s.step(2)
    s.sync()
    st = s.export_state()
    st["f"][0, 5, 777] = math.nan
    s.import_state(0, st)
    s.step(1)
    expect_error(s, LB_EUNSTABLE)
    s.close()


def test_fast_fluid_reports_unstable():
    """Fluid moving at |u| = 0.6 (beyond the 0.5 the kernels accept)."""
    from paper_1004_4414_gb300 import Simulation
    from paper_1004_4414_gb300.binding import LB_EUNSTABLE

    shape = (16, 12, 10)
    N = 16 * 12 * 10
    s = Simulation(dict(nx=16, ny=12, nz=10, n_particles=0, g_br=0.0, precision="fp32"))
    u = np.zeros((3, N))
    u[0] = 0.6
    s.init_fields(0, lbinputs.mixture(shape, amp=0.0), u=u)
    s.step(1)
    expect_error(s, LB_EUNSTABLE)
    s.close()


def test_fast_particle_reports_unstable():
    """A sphere given a velocity of 1.2 nodes per step."""
    from paper_1004_4414_gb300 import Simulation
    from paper_1004_4414_gb300.binding import LB_EUNSTABLE

    shape = (24, 24, 24)
    P = np.zeros((1, 9))
    P[0, 0:3] = (12.0, 12.0, 12.0)
    P[0, 3] = 1.2
    s = Simulation(dict(nx=24, ny=24, nz=24, n_particles=1, radius=3.0, g_br=0.0, precision="fp32",
                        particle_density=50.0))
    s.init_fields(0, lbinputs.mixture(shape, amp=0.0), particles=P)
    s.step(1)
    expect_error(s, LB_EUNSTABLE)
    s.close()


def test_neighbour_list_overflow():
    """Spheres of radius 0.6 on a grid of spacing 1.3: about 60 centres lie
    within the neighbour-list reach 2R + 2 of the middle one, more than the
    32 the list holds."""
    from paper_1004_4414_gb300 import Simulation
    from paper_1004_4414_gb300.binding import LB_EOVERFLOW

    shape = (24, 24, 24)
    g = np.arange(5) * 1.3 + 9.0
    X = np.array([(x, y, z) for x in g for y in g for z in g])
    P = np.zeros((len(X), 9))
    P[:, 0:3] = X
    s = Simulation(dict(nx=24, ny=24, nz=24, n_particles=len(X), radius=0.6, g_br=0.0, precision="fp32",
                        fixed_particles=1))
    s.init_fields(0, lbinputs.mixture(shape, amp=0.0), particles=P)
    s.step(1)
    expect_error(s, LB_EOVERFLOW)
    s.close()


def test_no_error_on_a_stable_run():
    from paper_1004_4414_gb300 import Simulation

    shape = (24, 20, 16)
    P = lbinputs.spheres(shape, 3.0, 3, seed=2, min_gap=1.0, vmax=0.02)
    s = Simulation(dict(nx=24, ny=20, nz=16, n_particles=3, radius=3.0, g_br=0.1, precision="fp32",
                        particle_density=2.0))
    s.init_fields(0, lbinputs.mixture(shape, amp=0.02, seed=4), particles=P)
    s.step(20)
    s.sync()
    assert s.observables()["error"] == 0
    s.close()
