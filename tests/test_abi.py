"""CPU checks of the C ABI: the library loads, exports every function that
include/lbpart.h declares, sizes workspaces and rejects invalid parameters
without touching a GPU."""
import ctypes as C
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbpart.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1004_4414_gb300 import build, binding

    build.build()
    return binding.load_library()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lb_[a-z_]+)\s*\(", src)))


def test_header_declares_the_abi():
    names = declared_functions()
    for f in ("lb_create", "lb_init_from_seed", "lb_step", "lb_observables", "lb_destroy"):
        assert f in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1004_4414_gb300 import binding

    names = declared_functions()
    assert set(names) == set(binding.ABI_FUNCTIONS)
    for name in names:
        assert hasattr(lib, name), name


def test_workspace_bytes_scale_with_precision(lib):
    from paper_1004_4414_gb300 import binding

    sizes = {}
    for prec in ("fp64", "fp32", "fp16", "bf16"):
        p = binding.make_params(nx=64, ny=64, nz=64, precision=prec)
        sizes[prec] = binding.workspace_bytes([p])
    N = 64 ** 3
    # populations dominate: 2 x 19 x 8 / 4 bytes, or 2 x 18 x 2 + 2 x 4 bytes
    assert sizes["fp64"] - sizes["fp32"] >= 2 * 19 * 4 * N
    assert sizes["fp16"] == sizes["bf16"]
    assert sizes["fp32"] - sizes["fp16"] >= (2 * 19 * 4 - 2 * 18 * 2 - 2 * 4) * N


def test_invalid_parameters_rejected(lib):
    from paper_1004_4414_gb300 import binding

    n = C.c_size_t(0)
    nan, inf = float("nan"), float("inf")
    for bad in (dict(nx=0), dict(tau=(0.5, 1.0)), dict(precision=7), dict(radius=0.0),
                dict(implicit_update=2), dict(implicit_update=1, aspect=1.5),
                dict(rho_init=(0.0, 0.7)), dict(lub_min=0.0), dict(lub_cut=0.1, lub_min=0.1),
                dict(aspect=0.05), dict(aspect=11.0), dict(aspect=-1.0), dict(aspect=nan),
                dict(ny=0), dict(nz=-3), dict(nx=65536), dict(nx=2048, ny=2048, nz=512),
                dict(tau=(1.0, 0.4)), dict(tau=(nan, 1.0)), dict(tau=(inf, 1.0)), dict(rho0=0.0),
                dict(rho0=inf), dict(particle_density=-1.0), dict(rho_init=(0.7, -0.1)),
                dict(rho_init=(inf, 0.7)), dict(vel_mode=2), dict(g_br=nan), dict(sc_weight=(1.0, inf)),
                dict(noise_amp=-0.01), dict(noise_amp=nan), dict(k_hertz=-1.0), dict(mass_corr_c0=-1.0),
                dict(color=nan), dict(body_force=(0.0, nan, 0.0)), dict(fixed_particles=2),
                dict(lub_cut=nan), dict(radius=inf),
                # a derived particle count must be a number of particles the box can hold
                dict(n_particles=-1, volume_fraction=nan), dict(n_particles=-1, volume_fraction=-0.1),
                dict(n_particles=-1, volume_fraction=1.0), dict(n_particles=-1, volume_fraction=1e30),
                dict(n_particles=-1, volume_fraction=0.5, radius=1e-4),
                dict(nx=4, ny=4, nz=4, n_particles=65)):
        p = binding.make_params(**bad)
        arr = (binding.LbParams * 1)(p)
        assert lib.lb_workspace_bytes(arr, 1, C.byref(n)) == binding.LB_EINVAL
    # spheres (aspect 0 or 1) and spheroids within [0.1, 10] are accepted; so
    # are an unused NaN volume fraction, a NaN contact angle (colour given)
    # and a box exactly full of particles by count
    for good in (dict(aspect=0.0), dict(aspect=1.0), dict(aspect=0.1), dict(aspect=10.0), dict(aspect=1.75),
                 dict(n_particles=3, volume_fraction=nan), dict(contact_angle_deg=nan, color=0.02),
                 dict(nx=4, ny=4, nz=4, n_particles=64), dict(n_particles=-1, volume_fraction=0.0)):
        arr = (binding.LbParams * 1)(binding.make_params(**good))
        assert lib.lb_workspace_bytes(arr, 1, C.byref(n)) == binding.LB_OK
    # a prolate spheroid needs a larger workspace than the sphere of its
    # equatorial radius (bounding-radius shell lists and event buffers)
    ws = []
    for a in (1.0, 2.0):
        arr = (binding.LbParams * 1)(binding.make_params(nx=64, ny=64, nz=64, n_particles=20, radius=4.0, aspect=a))
        assert lib.lb_workspace_bytes(arr, 1, C.byref(n)) == binding.LB_OK
        ws.append(n.value)
    assert ws[1] > ws[0]
    # mixed precisions in one batch are rejected
    arr = (binding.LbParams * 2)(binding.make_params(precision="fp32"), binding.make_params(precision="fp16"))
    assert lib.lb_workspace_bytes(arr, 2, C.byref(n)) == binding.LB_EINVAL
    # create without a workspace is rejected before any CUDA call
    h = C.c_void_p()
    arr = (binding.LbParams * 1)(binding.make_params())
    assert lib.lb_create(arr, 1, None, 0, None, C.byref(h)) == binding.LB_EINVAL
    # a misaligned or too small workspace and a missing handle pointer are
    # rejected from the arguments alone (the pointer is never dereferenced)
    assert lib.lb_workspace_bytes(arr, 1, C.byref(n)) == binding.LB_OK
    need = n.value
    assert lib.lb_create(arr, 1, C.c_void_p(0x100010), need, None, C.byref(h)) == binding.LB_EINVAL
    assert lib.lb_create(arr, 1, C.c_void_p(0x100000), need - 1, None, C.byref(h)) == binding.LB_ENOMEM
    assert lib.lb_create(arr, 1, C.c_void_p(0x100000), need, None, None) == binding.LB_EINVAL
    assert lib.lb_create(arr, 0, C.c_void_p(0x100000), need, None, C.byref(h)) == binding.LB_EINVAL
    assert not h.value
    assert lib.lb_step(None, 1) == binding.LB_EINVAL


def test_strerror(lib):
    assert lib.lb_strerror(0) == b"ok"
    assert b"unstable" in lib.lb_strerror(-4)


def test_params_struct_matches_header():
    """The ctypes mirror lists the header's lb_params fields in order."""
    from paper_1004_4414_gb300 import binding

    src = open(HEADER).read()
    body = src[src.index("typedef struct {"):src.index("} lb_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl or decl.startswith("typedef"):
            decl = decl.replace("typedef struct {", "").strip()
        if not decl:
            continue
        parts = decl.split(None, 1)
        for v in parts[1].split(","):
            names.append(re.sub(r"\[.*\]", "", v).strip())
    assert names == [f[0] for f in binding.LbParams._fields_]


def test_contact_angle_mapping_default_is_nan():
    from paper_1004_4414_gb300 import binding

    assert math.isnan(binding.make_params().contact_angle_deg)


def test_native_state_calls_reject_a_missing_handle(lib):
    """The storage-format state calls check their arguments before any CUDA
    call, and the binding's meta length is the header's LB_NATIVE_META."""
    from paper_1004_4414_gb300 import binding

    m = re.search(r"#define\s+LB_NATIVE_META\s+(\d+)", open(HEADER).read())
    assert m and int(m.group(1)) == binding.NATIVE_META
    n = C.c_size_t(0)
    meta = (C.c_double * binding.NATIVE_META)()
    assert lib.lb_state_native_bytes(None, 0, C.byref(n)) == binding.LB_EINVAL
    assert lib.lb_export_state_native(None, 0, None, 0, None, None, meta) == binding.LB_EINVAL
    assert lib.lb_import_state_native(None, 0, None, 0, None, None, meta) == binding.LB_EINVAL

