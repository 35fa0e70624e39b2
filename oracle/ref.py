"""ctypes wrapper around the FP64 CPU oracle (oracle/lbref.c).

Test infrastructure only.  Parameters are given as a dict whose keys are the
field names of ``orc_params``; missing keys take the defaults below, which
follow the paper's standard runs (tau = 1, g_br = 0.08, rho0 = 1,
R = 5, particle density 1, lubrication below a gap of 2/3 clamped at 1/10).
"""
import ctypes as C

import numpy as np

from . import build as _build

Q = 19


class OrcParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("n_particles", C.c_int32),
        ("tau", C.c_double * 2),
        ("g_br", C.c_double),
        ("rho0", C.c_double),
        ("sc_weight", C.c_double * 2),
        ("rho_init", C.c_double * 2),
        ("noise_amp", C.c_double),
        ("volume_fraction", C.c_double),
        ("radius", C.c_double),
        ("particle_density", C.c_double),
        ("color", C.c_double),
        ("k_hertz", C.c_double),
        ("lub_cut", C.c_double),
        ("lub_min", C.c_double),
        ("mass_corr_c0", C.c_double),
        ("body_force", C.c_double * 3),
        ("vel_mode", C.c_int32),
        ("virtual_fluid", C.c_int32),
        ("fixed_particles", C.c_int32),
        ("pad_", C.c_int32),
        ("seed", C.c_uint64),
        ("aspect", C.c_double),
        ("implicit_update", C.c_int32),
        ("pad2_", C.c_int32),
    ]


class OrcObs(C.Structure):
    _fields_ = [
        ("step", C.c_int64),
        ("mass", C.c_double * 2),
        ("mom_fluid", C.c_double * 3),
        ("mom_part", C.c_double * 3),
        ("max_u", C.c_double),
        ("n_cover", C.c_int64),
        ("n_uncover", C.c_int64),
    ]


DEFAULTS = dict(
    nx=16, ny=16, nz=16, n_particles=0, tau=(1.0, 1.0), g_br=0.08, rho0=1.0,
    sc_weight=(2.0, 1.0), rho_init=(0.7, 0.7), noise_amp=0.01, volume_fraction=0.0,
    radius=5.0, particle_density=1.0, color=0.0, k_hertz=100.0, lub_cut=2.0 / 3.0,
    lub_min=0.1, mass_corr_c0=0.0, body_force=(0.0, 0.0, 0.0), vel_mode=0,
    virtual_fluid=1, fixed_particles=0, seed=1, aspect=1.0, implicit_update=0,
)

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int32)
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(OrcParams), C.c_int32]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_n_particles.argtypes = [C.c_void_p]
        L.orc_n_particles.restype = C.c_int32
        L.orc_init_from_seed.argtypes = [C.c_void_p, C.c_uint64]
        L.orc_init_fields.argtypes = [C.c_void_p, dp, dp, dp, ip]
        L.orc_step.argtypes = [C.c_void_p, C.c_int32]
        L.orc_get_state.argtypes = [C.c_void_p, dp, ip, dp, dp]
        L.orc_set_state.argtypes = [C.c_void_p, dp, ip, dp, dp]
        L.orc_get_rho.argtypes = [C.c_void_p, dp]
        L.orc_get_forces.argtypes = [C.c_void_p, dp, dp]
        L.orc_set_particle_colors.argtypes = [C.c_void_p, dp]
        L.orc_observe.argtypes = [C.c_void_p, C.POINTER(OrcObs)]
        L.orc_last_psi.argtypes = [C.c_void_p, dp]
        L.orc_last_sc_force.argtypes = [C.c_void_p, dp]
        L.orc_feq.argtypes = [C.c_double, dp, dp]
        L.orc_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
        L.orc_splitmix64.restype = C.c_uint64
        L.orc_unit.argtypes = [C.c_uint64, C.c_uint64]
        L.orc_unit.restype = C.c_double
        L.orc_lattice.argtypes = [C.c_void_p, dp, ip]
        L.orc_set_threads.argtypes = [C.c_int32]
        L.orc_pair_force.argtypes = [C.POINTER(OrcParams), dp, dp, dp, dp, dp]
        L.orc_debug_remap.argtypes = [C.c_void_p]
        L.orc_get_axes.argtypes = [C.c_void_p, dp]
        L.orc_set_axes.argtypes = [C.c_void_p, dp]
        L.orc_inside.argtypes = [C.POINTER(OrcParams), dp, dp]
        L.orc_inside.restype = C.c_int32
        L.orc_contact_distance.argtypes = [C.POINTER(OrcParams), dp, dp, dp]
        L.orc_contact_distance.restype = C.c_double
        L.orc_rotate.argtypes = [C.POINTER(OrcParams), dp, dp, dp]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def make_params(**kw):
    d = dict(DEFAULTS)
    unknown = set(kw) - set(d)
    if unknown:
        raise KeyError("unknown oracle parameters: %s" % sorted(unknown))
    d.update(kw)
    p = OrcParams()
    for k, v in d.items():
        if isinstance(v, (tuple, list)):
            arr = getattr(p, k)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(p, k, v)
    return p


def lattice():
    c = np.zeros((19, 3), np.int32)
    w = np.zeros(19)
    opp = np.zeros(19, np.int32)
    lib().orc_lattice(c.ctypes.data_as(C.c_void_p), _dp(w), _ip(opp))
    return c, w, opp


def feq(rho, u):
    out = np.zeros(19)
    uu = np.ascontiguousarray(u, dtype=np.float64)
    lib().orc_feq(float(rho), _dp(uu), _dp(out))
    return out


def splitmix64(seed, n):
    return int(lib().orc_splitmix64(seed, n))


def unit(seed, n):
    return float(lib().orc_unit(seed, n))


def pair_force(Xp, Xq, Up, Uq, **params):
    """Hertz + lubrication force on particle p from particle q."""
    P = make_params(**params)
    a = [np.ascontiguousarray(v, np.float64) for v in (Xp, Xq, Up, Uq)]
    out = np.zeros(3)
    lib().orc_pair_force(C.byref(P), *[_dp(v) for v in a], _dp(out))
    return out


def inside(d, e, **params):
    """Inside test of displacement d for a particle with body axis e."""
    P = make_params(**params)
    dd, ee = np.ascontiguousarray(d, np.float64), np.ascontiguousarray(e, np.float64)
    return bool(lib().orc_inside(C.byref(P), _dp(dd), _dp(ee)))


def contact_distance(rh, ep, eq, **params):
    P = make_params(**params)
    a = [np.ascontiguousarray(v, np.float64) for v in (rh, ep, eq)]
    return float(lib().orc_contact_distance(C.byref(P), *[_dp(v) for v in a]))


def rotate(W, e, T, **params):
    """One rotational MD update of a free particle; returns (omega, e)."""
    P = make_params(**params)
    W = np.array(W, np.float64)
    e = np.array(e, np.float64)
    T = np.ascontiguousarray(T, np.float64)
    lib().orc_rotate(C.byref(P), _dp(W), _dp(e), _dp(T))
    return W, e


def set_threads(n):
    lib().orc_set_threads(int(n))


class Oracle:
    """One periodic box stepped by the FP64 reference."""

    def __init__(self, **params):
        self.params = make_params(**params)
        self._h = lib().orc_create(C.byref(self.params), int(self.params.n_particles))
        if not self._h:
            raise ValueError("oracle rejected the parameters")
        self.nx, self.ny, self.nz = self.params.nx, self.params.ny, self.params.nz
        self.N = self.nx * self.ny * self.nz
        self.np = lib().orc_n_particles(self._h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    # -- init -----------------------------------------------------------
    def init_from_seed(self, seed):
        rc = lib().orc_init_from_seed(self._h, seed)
        if rc != 0:
            raise RuntimeError("oracle seeded init failed (%d)" % rc)

    def init_fields(self, rho, u=None, particles=None, walls=None):
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(2, self.N)
        up = None if u is None else np.ascontiguousarray(u, np.float64).reshape(3, self.N)
        parts = np.zeros((max(self.np, 1), 9)) if particles is None else \
            np.ascontiguousarray(particles, np.float64).reshape(-1, 9)
        if parts.shape[0] < self.np:
            raise ValueError("need %d particles" % self.np)
        wl = None if walls is None else np.ascontiguousarray(walls, np.int32).reshape(self.N)
        lib().orc_init_fields(self._h, _dp(rho), None if up is None else _dp(up), _dp(parts),
                              None if wl is None else _ip(wl))

    # -- stepping -------------------------------------------------------
    def step(self, n=1):
        lib().orc_step(self._h, int(n))

    def debug_remap(self):
        """Run only the particle remap (cover/uncover) of the next step."""
        lib().orc_debug_remap(self._h)

    # -- state ----------------------------------------------------------
    def get_state(self):
        f = np.zeros((2, Q, self.N))
        owner = np.zeros(self.N, np.int32)
        parts = np.zeros((max(self.np, 1), 9))
        meta = np.zeros(4)
        lib().orc_get_state(self._h, _dp(f), _ip(owner), _dp(parts), _dp(meta))
        return dict(f=f, owner=owner, particles=parts[: self.np], meta=meta)

    def set_state(self, st):
        f = np.ascontiguousarray(st["f"], np.float64)
        owner = np.ascontiguousarray(st["owner"], np.int32)
        parts = np.ascontiguousarray(st["particles"], np.float64).reshape(-1, 9)
        if parts.shape[0] == 0:
            parts = np.zeros((1, 9))
        meta = np.ascontiguousarray(st["meta"], np.float64)
        lib().orc_set_state(self._h, _dp(f), _ip(owner), _dp(parts), _dp(meta))

    def rho(self):
        r = np.zeros((2, self.N))
        lib().orc_get_rho(self._h, _dp(r))
        return r

    def particle_forces(self):
        F = np.zeros((max(self.np, 1), 3))
        T = np.zeros((max(self.np, 1), 3))
        lib().orc_get_forces(self._h, _dp(F), _dp(T))
        return F[: self.np], T[: self.np]

    def axes(self):
        e = np.zeros((max(self.np, 1), 3))
        lib().orc_get_axes(self._h, _dp(e))
        return e[: self.np]

    def set_axes(self, e):
        ee = np.ascontiguousarray(e, np.float64).reshape(-1, 3)
        lib().orc_set_axes(self._h, _dp(ee))

    def set_colors(self, colors):
        col = np.ascontiguousarray(colors, np.float64)
        lib().orc_set_particle_colors(self._h, _dp(col))

    def last_psi(self):
        p = np.zeros((2, self.N))
        lib().orc_last_psi(self._h, _dp(p))
        return p

    def last_sc_force(self):
        F = np.zeros((2, 3, self.N))
        lib().orc_last_sc_force(self._h, _dp(F))
        return F

    def observe(self):
        o = OrcObs()
        lib().orc_observe(self._h, C.byref(o))
        return dict(step=o.step, mass=np.array(o.mass[:]), mom_fluid=np.array(o.mom_fluid[:]),
                    mom_part=np.array(o.mom_part[:]), max_u=o.max_u,
                    n_cover=o.n_cover, n_uncover=o.n_uncover)

    def phi(self):
        """Order parameter rho^r - rho^b, 0 on solid nodes (shape nz, ny, nx)."""
        r = self.rho()
        return (r[0] - r[1]).reshape(self.nz, self.ny, self.nx)

    def velocity(self):
        """Total fluid velocity j / rho per node, 0 on solid (shape 3, N)."""
        st = self.get_state()
        c, _, _ = lattice()
        f = st["f"]
        rho = f.sum(axis=(0, 1))
        j = np.einsum("cin,ia->an", f, c.astype(np.float64))
        with np.errstate(invalid="ignore", divide="ignore"):
            u = np.where(rho > 0, j / np.where(rho > 0, rho, 1.0), 0.0)
        return u
