"""The storage-format state (lb_export_state_native / lb_import_state_native).

The format is the device's own bytes: the 18 stored population pairs of
every node in the in-place streaming order of the current step, then the
density field.  Checked here:
- a round trip through a fresh handle returns every byte, and the FP64
  canonical export of the importing handle equals the exporter's bit for
  bit, in every storage and at both step parities;
- a run continued from the imported bytes follows the FP64 oracle run from
  the same seeded start (moving, rotating spheres with cover / uncover
  events and mass correction), to the FP64 parity tolerance;
- in FP32 storage, the continued run stays with the uninterrupted one to
  the FP32 parity tolerance (the two differ only in the summation order of
  the particle forces, since the import rebuilds the shell lists);
- the same for the uneven boxes of one batched handle (box-local particle
  indices in the owner map);
- a byte count, storage type or node count that does not match, an owner
  entry out of range, and an export before any init are rejected, the
  first four before anything of the box changes.
"""
import numpy as np
import pytest

import lbinputs
from oracle import ref

pytestmark = pytest.mark.gpu

SHAPE = (26, 22, 20)
BYTES_PER_NODE = {"fp64": 18 * 16 + 16, "fp32": 18 * 8 + 8, "fp16": 18 * 4 + 8, "bf16": 18 * 4 + 8}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1004_4414_gb300 import build

    build.build()
    ref.lib()


def params(precision):
    nx, ny, nz = SHAPE
    return dict(nx=nx, ny=ny, nz=nz, n_particles=5, radius=3.3, g_br=0.12, color=-0.03, particle_density=3.0,
                mass_corr_c0=5.0, precision=precision)


def seeded():
    P = lbinputs.spheres(SHAPE, 3.3, 5, seed=12, min_gap=0.4, vmax=0.06, wmax=0.03)
    rho = lbinputs.mixture(SHAPE, amp=0.05, seed=13)
    return rho, P


def started(precision, steps):
    from paper_1004_4414_gb300 import Simulation

    rho, P = seeded()
    s = Simulation(params(precision))
    s.init_fields(0, rho, particles=P)
    s.step(steps)
    return s


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16", "bf16"])
@pytest.mark.parametrize("steps", [7, 8])
def test_roundtrip_returns_every_byte(precision, steps):
    from paper_1004_4414_gb300 import Simulation

    a = started(precision, steps)
    n = a.export_state_native()
    c = a.export_state()
    N = int(np.prod(SHAPE))
    assert n["state"].size == BYTES_PER_NODE[precision] * N
    assert n["meta"][0] == steps and n["meta"][5] == N
    b = Simulation(params(precision))
    b.import_state_native(0, n)
    n2 = b.export_state_native()
    assert np.array_equal(n2["state"], n["state"])
    assert np.array_equal(n2["owner"], n["owner"])
    assert np.array_equal(n2["particles"], n["particles"])
    assert np.array_equal(n2["meta"], n["meta"])
    c2 = b.export_state()
    assert np.array_equal(c2["f"], c["f"])
    assert np.array_equal(c2["owner"], c["owner"])
    assert np.array_equal(c2["particles"], c["particles"])
    assert b.observables()["error"] == 0


@pytest.mark.parametrize("steps", [7, 8])
def test_continued_run_follows_the_oracle_fp64(steps):
    from paper_1004_4414_gb300 import Simulation

    nx, ny, nz = SHAPE
    rho, P = seeded()
    o = ref.Oracle(nx=nx, ny=ny, nz=nz, n_particles=5, radius=3.3, g_br=0.12, color=-0.03, particle_density=3.0,
                   mass_corr_c0=5.0)
    o.init_fields(rho, particles=P)
    a = started("fp64", steps)
    b = Simulation(params("fp64"))
    b.import_state_native(0, a.export_state_native())
    o.step(steps + 12)
    b.step(12)
    got, want = b.export_state(), o.get_state()
    assert np.array_equal(got["owner"], want["owner"])
    assert np.max(np.abs(got["f"] - want["f"])) < 1e-11
    assert np.max(np.abs(got["particles"] - want["particles"])) < 1e-11
    ob, sb = o.observe(), b.observables()
    assert np.allclose(ob["mass"], sb["mass"], rtol=1e-13)


def test_continued_run_follows_the_uninterrupted_one_fp32():
    from paper_1004_4414_gb300 import Simulation

    a = started("fp32", 9)
    b = Simulation(params("fp32"))
    b.import_state_native(0, a.export_state_native())
    a.step(20)
    b.step(20)
    x, y = a.export_state(), b.export_state()
    assert np.array_equal(x["owner"], y["owner"])
    scale = np.maximum(np.abs(x["f"]), 1e-3)
    assert np.max(np.abs(x["f"] - y["f"]) / scale) < 1e-5
    assert np.max(np.abs(x["particles"] - y["particles"])) < 1e-6


def test_mismatches_rejected_without_changes():
    from paper_1004_4414_gb300 import Simulation, binding

    a = started("fp32", 5)
    n = a.export_state_native()
    b = started("fp32", 5)
    b.step(3)
    before = b.export_state_native()
    bad_cases = []
    bad_cases.append(dict(n, state=n["state"][:-16].copy()))  # byte count
    m = n["meta"].copy()
    m[4] = binding.LB_FP16_DEV  # storage type
    bad_cases.append(dict(n, meta=m))
    m = n["meta"].copy()
    m[5] += 1  # node count
    bad_cases.append(dict(n, meta=m))
    o = n["owner"].copy()
    o[11] = 7  # no particle 7 in this box
    bad_cases.append(dict(n, owner=o))
    for bad in bad_cases:
        with pytest.raises(binding.LbError) as e:
            b.import_state_native(0, bad)
        assert e.value.code == binding.LB_EINVAL
        after = b.export_state_native()
        assert np.array_equal(after["state"], before["state"])
        assert np.array_equal(after["owner"], before["owner"])
        assert np.array_equal(after["particles"], before["particles"])
    # a fresh handle has no state to export
    c = Simulation(params("fp32"))
    with pytest.raises(binding.LbError) as e:
        c.export_state_native()
    assert e.value.code == binding.LB_EINVAL


@pytest.mark.parametrize("precision", ["fp64", "fp16"])
def test_batched_boxes_roundtrip(precision):
    """Uneven boxes of one handle: each box's storage-format state (with
    box-local particle indices in the owner map) returns every byte through
    a second handle at the shared step, and the continued batch follows the
    FP64 oracle box by box."""
    from paper_1004_4414_gb300 import Simulation

    specs = [dict(nx=16, ny=16, nz=16, n_particles=2, radius=3.0, color=0.03),
             dict(nx=24, ny=20, nz=12, n_particles=3, radius=2.5, color=-0.02, g_br=0.1),
             dict(nx=12, ny=12, nz=20, n_particles=0)]
    mk = lambda: Simulation([dict(sp, precision=precision, particle_density=2.0) for sp in specs])
    a, b = mk(), mk()
    oracles = []
    for k, sp in enumerate(specs):
        shape = (sp["nx"], sp["ny"], sp["nz"])
        P = lbinputs.spheres(shape, sp.get("radius", 5.0), sp["n_particles"], seed=50 + k, min_gap=0.5,
                             vmax=0.04, wmax=0.02) if sp["n_particles"] else None
        rho = lbinputs.mixture(shape, amp=0.04, seed=60 + k)
        o = ref.Oracle(**dict(sp, particle_density=2.0))
        o.init_fields(rho, particles=P)
        oracles.append(o)
        a.init_fields(k, rho, particles=P)
        b.init_fields(k, rho, particles=P)
    a.step(5)
    b.step(5)
    states = [a.export_state_native(k) for k in range(len(specs))]
    assert max(int(np.max(st["owner"])) for st in states) < 3  # box-local indices
    for k, st in enumerate(states):
        b.import_state_native(k, st)
    for k, st in enumerate(states):
        back = b.export_state_native(k)
        assert np.array_equal(back["state"], st["state"])
        assert np.array_equal(back["owner"], st["owner"])
        assert np.array_equal(back["particles"], st["particles"])
        assert np.array_equal(b.export_state(k)["owner"], a.export_state(k)["owner"])
    if precision == "fp64":
        for o in oracles:
            o.step(15)
        b.step(10)
        for k, o in enumerate(oracles):
            got, want = b.export_state(k), o.get_state()
            assert np.array_equal(got["owner"], want["owner"])
            assert np.max(np.abs(got["f"] - want["f"])) < 1e-11
            if want["particles"].size:
                assert np.max(np.abs(got["particles"] - want["particles"])) < 1e-11
