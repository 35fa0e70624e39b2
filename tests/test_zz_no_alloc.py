"""lb_field_moments (field sums without allocating, scratch held by the
library) against lb_observables on the same state.

The file sorts last so that it also runs after every other test has used the
library and the device; it must pass alone in a fresh process as well."""
import numpy as np
import pytest


def _lib():
    from paper_1004_4414_gb300 import binding, build

    build.build()
    return binding, binding.load_library()


def test_field_moments_rejects_sizes_beyond_the_maximum():
    # rejected on the host before any device call, so this runs without a GPU
    binding, L = _lib()
    assert L.lb_field_moments(None, None, binding.FIELD_MOMENTS_MAX_NODES + 1, None, None) == binding.LB_EINVAL
    assert L.lb_field_moments(None, None, -1, None, None) == binding.LB_EINVAL


def _check(binding, sim, out):
    import torch

    ob = sim.observables()
    assert ob["error"] == 0
    st = sim.export_state(0)
    f = torch.from_numpy(st["f"]).to(out.device)
    owner = torch.from_numpy(st["owner"]).to(out.device)
    out.fill_(float("nan"))
    binding.field_moments(f, owner, out)
    torch.cuda.synchronize()
    v = out.cpu().numpy()
    mass = ob["mass"]
    # FP64 sums in a different order than lb_observables: 1e-12 relative
    np.testing.assert_allclose(v[0:2], mass, rtol=1e-12, atol=0)
    np.testing.assert_allclose(v[2:5], ob["mom_fluid"], rtol=0, atol=1e-12 * mass.sum())
    np.testing.assert_allclose(v[5], ob["max_u"], rtol=1e-12, atol=0)
    assert v[6] == ob["n_fluid"] and v[7] == ob["n_solid"]
    assert ob["n_fluid"] + ob["n_solid"] == owner.numel()
    # and against plain NumPy sums of the exported populations
    fl = st["owner"] == -1
    ff = st["f"][:, :, fl]
    c = np.array([[0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0],
                  [0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1],
                  [0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1]], float)
    np.testing.assert_allclose(v[0:2], ff.sum(axis=(1, 2)), rtol=1e-12, atol=0)
    j = np.einsum("ai,cin->an", c, ff)
    np.testing.assert_allclose(v[2:5], j.sum(axis=1), rtol=0, atol=1e-12 * mass.sum())
    np.testing.assert_allclose(v[5], np.max(np.linalg.norm(j, axis=0) / ff.sum(axis=(0, 1))), rtol=1e-12)
    assert v[6] == fl.sum() and v[7] == (~fl).sum()
    return v


@pytest.mark.gpu
def test_field_moments_matches_observables_on_two_calls_in_a_row():
    import torch
    from paper_1004_4414_gb300 import Simulation

    binding, _ = _lib()
    out = torch.empty(8, dtype=torch.float64, device="cuda")
    base = dict(n_particles=6, radius=4.0, rho_init=(0.42, 0.28), color=-0.03)
    # first call: 163,840 nodes -> 640 blocks of the scratch
    big = Simulation(dict(base, nx=64, ny=64, nz=40))
    big.init_from_seed(11)
    big.step(9)
    v1 = _check(binding, big, out)
    big.close()
    # second call: 47,520 nodes -> 186 blocks, the last one ragged; the
    # partials the first call left in blocks 186..639 must not leak in
    small = Simulation(dict(base, nx=40, ny=36, nz=33))
    small.init_from_seed(12)
    small.step(14)
    v2 = _check(binding, small, out)
    small.close()
    assert v1[6] + v1[7] == 64 * 64 * 40 and v2[6] + v2[7] == 40 * 36 * 33
