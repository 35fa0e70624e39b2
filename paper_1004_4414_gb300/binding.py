"""Thin Python binding of the C ABI in include/lbpart.h (argument marshalling
only; every step of the method runs in the library's sm_103a kernels).

PyTorch provides the device workspace (one uint8 tensor the library lays
its arrays out in) and the CUDA stream.  The shared library must have been
built (``paper_1004_4414_gb300.build.build()``); importing it fails loudly
otherwise -- there is no CPU fallback.
"""
import ctypes as C
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liblbpart.so")

LB_OK, LB_EINVAL, LB_ENOMEM, LB_ECUDA, LB_EUNSTABLE, LB_EPLACE, LB_ETIMEOUT, LB_EOVERFLOW = 0, -1, -2, -3, -4, -5, -6, -7
LB_FP64, LB_FP32, LB_FP16_DEV, LB_BF16_DEV = 0, 1, 2, 3
PRECISIONS = {"fp64": LB_FP64, "fp32": LB_FP32, "fp16": LB_FP16_DEV, "bf16": LB_BF16_DEV}
NATIVE_META = 8  # LB_NATIVE_META


class LbParams(C.Structure):
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
        ("contact_angle_deg", C.c_double),
        ("k_hertz", C.c_double),
        ("lub_cut", C.c_double),
        ("lub_min", C.c_double),
        ("mass_corr_c0", C.c_double),
        ("body_force", C.c_double * 3),
        ("vel_mode", C.c_int32),
        ("fixed_particles", C.c_int32),
        ("precision", C.c_int32),
        ("implicit_update", C.c_int32),
        ("aspect", C.c_double),
    ]


class LbObs(C.Structure):
    _fields_ = [
        ("step", C.c_int64),
        ("mass", C.c_double * 2),
        ("mom_fluid", C.c_double * 3),
        ("mom_part", C.c_double * 3),
        ("max_u", C.c_double),
        ("n_cover", C.c_int64),
        ("n_uncover", C.c_int64),
        ("n_fluid", C.c_int64),
        ("n_solid", C.c_int64),
        ("error", C.c_int32),
        ("n_particles", C.c_int32),
        ("L", C.c_double * 3),
        ("coverage", C.c_double),
    ]


# Defaults follow the paper's runs: tau = 1, g_br = 0.08, rho0 = 1, R = 5,
# particle density 1, lubrication below a gap of 2/3 clamped at 1/10.
DEFAULTS = dict(
    nx=32, ny=32, nz=32, n_particles=0, tau=(1.0, 1.0), g_br=0.08, rho0=1.0,
    sc_weight=(2.0, 1.0), rho_init=(0.7, 0.7), noise_amp=0.01, volume_fraction=0.0,
    radius=5.0, particle_density=1.0, color=0.0, contact_angle_deg=math.nan,
    k_hertz=100.0, lub_cut=2.0 / 3.0, lub_min=0.1, mass_corr_c0=0.0,
    body_force=(0.0, 0.0, 0.0), vel_mode=0, fixed_particles=0, precision=LB_FP32, implicit_update=0, aspect=1.0,
)

ABI_FUNCTIONS = (
    "lb_workspace_bytes", "lb_create", "lb_init_from_seed", "lb_init_fields", "lb_step", "lb_sync",
    "lb_observables", "lb_export_state", "lb_import_state", "lb_state_native_bytes", "lb_export_state_native",
    "lb_import_state_native", "lb_export_rho", "lb_export_phi",
    "lb_set_particle_colors",
    "lb_set_axes", "lb_get_axes",
    "lb_particle_forces", "lb_box_info", "lb_set_tiling", "lb_set_profiling", "lb_kernel_time", "lb_phase_times",
    "lb_destroy", "lb_strerror", "lb_field_moments",
)

_lib = None


class LbError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s failed: %s (%d)" % (where, strerror(code), code))


def load_library(path=LIB_PATH):
    """Load the shared library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("CUDA library %s is missing: run paper_1004_4414_gb300.build.build()" % path)
    L = C.CDLL(path)
    vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32)
    P = C.POINTER(LbParams)
    L.lb_workspace_bytes.argtypes = [P, C.c_int32, C.POINTER(C.c_size_t)]
    L.lb_create.argtypes = [P, C.c_int32, vp, C.c_size_t, vp, C.POINTER(vp)]
    L.lb_init_from_seed.argtypes = [vp, C.c_uint64]
    L.lb_init_fields.argtypes = [vp, C.c_int32, dp, dp, dp, ip]
    L.lb_step.argtypes = [vp, C.c_int64]
    L.lb_sync.argtypes = [vp]
    L.lb_observables.argtypes = [vp, C.c_int32, C.POINTER(LbObs)]
    L.lb_export_state.argtypes = [vp, C.c_int32, dp, ip, dp, dp]
    L.lb_import_state.argtypes = [vp, C.c_int32, dp, ip, dp, dp]
    L.lb_state_native_bytes.argtypes = [vp, C.c_int32, C.POINTER(C.c_size_t)]
    L.lb_export_state_native.argtypes = [vp, C.c_int32, vp, C.c_size_t, ip, dp, dp]
    L.lb_import_state_native.argtypes = [vp, C.c_int32, vp, C.c_size_t, ip, dp, dp]
    L.lb_export_rho.argtypes = [vp, C.c_int32, dp]
    L.lb_export_phi.argtypes = [vp, C.c_int32, dp, dp, dp]
    L.lb_set_particle_colors.argtypes = [vp, C.c_int32, dp]
    L.lb_set_axes.argtypes = [vp, C.c_int32, dp]
    L.lb_get_axes.argtypes = [vp, C.c_int32, dp]
    L.lb_particle_forces.argtypes = [vp, C.c_int32, dp, dp]
    L.lb_box_info.argtypes = [vp, C.c_int32, ip, C.POINTER(C.c_int64)]
    L.lb_set_tiling.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32]
    L.lb_set_profiling.argtypes = [vp, C.c_int32]
    L.lb_kernel_time.argtypes = [vp, dp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    L.lb_phase_times.argtypes = [vp, dp, C.c_int32]
    L.lb_destroy.argtypes = [vp]
    L.lb_destroy.restype = None
    L.lb_strerror.argtypes = [C.c_int]
    L.lb_strerror.restype = C.c_char_p
    L.lb_field_moments.argtypes = [vp, vp, C.c_int64, vp, vp]
    _lib = L
    return L


def strerror(code):
    if _lib is None:
        return "error"
    return _lib.lb_strerror(code).decode()


def _ck(rc, where):
    if rc != LB_OK:
        raise LbError(rc, where)


FIELD_MOMENTS_MAX_NODES = 1 << 27


def field_moments(f, owner, out, stream=None):
    """lb_field_moments on torch CUDA tensors, without allocating: f float64
    (2, 19, N) and owner int32 (N,) in the lb_export_state layout, out a
    float64 tensor of 8 values on the same device ({mass_r, mass_b, j_x, j_y,
    j_z, max |u|, n_fluid, n_solid}).  Asynchronous on `stream` (default: the
    current torch stream)."""
    import torch

    n = owner.numel()
    if f.dtype != torch.float64 or owner.dtype != torch.int32 or out.dtype != torch.float64:
        raise TypeError("f and out must be float64, owner int32")
    if f.numel() != 2 * 19 * n or out.numel() < 8 or not (f.is_contiguous() and owner.is_contiguous()):
        raise ValueError("f must be contiguous (2, 19, N) for owner of N nodes; out needs 8 values")
    if not (f.device == owner.device == out.device) or out.device.type != "cuda":
        raise ValueError("f, owner and out must be on the same CUDA device")
    # the library checks the pointers against the current device
    with torch.cuda.device(out.device):
        s = stream if stream is not None else torch.cuda.current_stream(out.device)
        _ck(load_library().lb_field_moments(C.c_void_p(f.data_ptr()), C.c_void_p(owner.data_ptr()), n,
                                            C.c_void_p(s.cuda_stream), C.c_void_p(out.data_ptr())),
            "lb_field_moments")
    return out


def make_params(**kw):
    d = dict(DEFAULTS)
    unknown = set(kw) - set(d)
    if unknown:
        raise KeyError("unknown parameters: %s" % sorted(unknown))
    d.update(kw)
    if isinstance(d["precision"], str):
        d["precision"] = PRECISIONS[d["precision"]]
    p = LbParams()
    for k, v in d.items():
        if isinstance(v, (tuple, list)):
            arr = getattr(p, k)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(p, k, v)
    return p


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def workspace_bytes(boxes):
    L = load_library()
    arr = (LbParams * len(boxes))(*boxes)
    n = C.c_size_t(0)
    _ck(L.lb_workspace_bytes(arr, len(boxes), C.byref(n)), "lb_workspace_bytes")
    return n.value


class Simulation:
    """A batch of periodic boxes stepped together on one GPU.

    boxes: a dict of parameters (one box) or a list of dicts.
    """

    def __init__(self, boxes, device=None, stream=None):
        import torch

        L = load_library()
        if isinstance(boxes, dict):
            boxes = [boxes]
        self._params = [make_params(**b) for b in boxes]
        self.nb = len(self._params)
        arr = (LbParams * self.nb)(*self._params)
        n = C.c_size_t(0)
        _ck(L.lb_workspace_bytes(arr, self.nb, C.byref(n)), "lb_workspace_bytes")
        self.device = torch.device(device or "cuda")
        self.workspace = torch.empty(n.value + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        self._ws = base + (-base) % 256
        # a stream of its own: CUDA graphs cannot be captured on the legacy
        # default stream
        self.stream = stream or torch.cuda.Stream(self.device)
        h = C.c_void_p()
        _ck(L.lb_create(arr, self.nb, C.c_void_p(self._ws), n.value, C.c_void_p(self.stream.cuda_stream),
                        C.byref(h)), "lb_create")
        self._h = h
        self.dims = [(p.nx, p.ny, p.nz) for p in self._params]
        self.n_particles = []
        self.n_nodes = []
        for b in range(self.nb):
            npart, nn = C.c_int32(0), C.c_int64(0)
            _ck(L.lb_box_info(self._h, b, C.byref(npart), C.byref(nn)), "lb_box_info")
            self.n_particles.append(npart.value)
            self.n_nodes.append(nn.value)

    def close(self):
        if getattr(self, "_h", None):
            load_library().lb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- initial state ------------------------------------------------------
    def init_from_seed(self, seed):
        _ck(load_library().lb_init_from_seed(self._h, int(seed)), "lb_init_from_seed")

    def init_fields(self, box, rho, u=None, particles=None, walls=None):
        N = self.n_nodes[box]
        rho = np.ascontiguousarray(rho, np.float64).reshape(2, N)
        up = None if u is None else np.ascontiguousarray(u, np.float64).reshape(3, N)
        npb = self.n_particles[box]
        parts = np.zeros((max(npb, 1), 9)) if particles is None else \
            np.ascontiguousarray(particles, np.float64).reshape(-1, 9)
        wl = None if walls is None else np.ascontiguousarray(walls, np.int32).reshape(N)
        _ck(load_library().lb_init_fields(self._h, box, _dp(rho), None if up is None else _dp(up), _dp(parts),
                                          None if wl is None else _ip(wl)), "lb_init_fields")

    # -- stepping -------------------------------------------------------------
    def step(self, n=1):
        _ck(load_library().lb_step(self._h, int(n)), "lb_step")

    def sync(self):
        _ck(load_library().lb_sync(self._h), "lb_sync")

    # -- state ------------------------------------------------------------------
    def observables(self, box=0):
        o = LbObs()
        _ck(load_library().lb_observables(self._h, box, C.byref(o)), "lb_observables")
        return dict(step=o.step, mass=np.array(o.mass[:]), mom_fluid=np.array(o.mom_fluid[:]),
                    mom_part=np.array(o.mom_part[:]), max_u=o.max_u, n_cover=o.n_cover,
                    n_uncover=o.n_uncover, n_fluid=o.n_fluid, n_solid=o.n_solid, error=o.error,
                    n_particles=o.n_particles, L=np.array(o.L[:]), coverage=o.coverage)

    def export_state(self, box=0, f=True, f_out=None, owner_out=None):
        """Canonical state; f_out / owner_out: optional C-contiguous float64
        (2, 19, N) / int32 (N,) arrays to fill (e.g. pinned host memory)."""
        N = self.n_nodes[box]
        if f_out is not None:
            if f_out.dtype != np.float64 or f_out.size != 2 * 19 * N or not f_out.flags.c_contiguous:
                raise ValueError("f_out must be a C-contiguous float64 array of 2*19*N values")
            fa = f_out
        else:
            fa = np.zeros((2, 19, N)) if f else None
        if owner_out is not None:
            if owner_out.dtype != np.int32 or owner_out.size != N or not owner_out.flags.c_contiguous:
                raise ValueError("owner_out must be a C-contiguous int32 array of N values")
            owner = owner_out
        else:
            owner = np.zeros(N, np.int32)
        parts = np.zeros((max(self.n_particles[box], 1), 9))
        meta = np.zeros(4)
        _ck(load_library().lb_export_state(self._h, box, None if fa is None else _dp(fa), _ip(owner), _dp(parts),
                                           _dp(meta)), "lb_export_state")
        return dict(f=fa, owner=owner, particles=parts[: self.n_particles[box]], meta=meta)

    def import_state(self, box, st):
        f = np.ascontiguousarray(st["f"], np.float64)
        owner = np.ascontiguousarray(st["owner"], np.int32)
        parts = np.ascontiguousarray(st["particles"], np.float64).reshape(-1, 9)
        if parts.shape[0] == 0:
            parts = np.zeros((1, 9))
        meta = np.ascontiguousarray(st["meta"], np.float64)
        _ck(load_library().lb_import_state(self._h, box, _dp(f), _ip(owner), _dp(parts), _dp(meta)),
            "lb_import_state")

    def native_bytes(self, box=0):
        n = C.c_size_t(0)
        _ck(load_library().lb_state_native_bytes(self._h, box, C.byref(n)), "lb_state_native_bytes")
        return n.value

    def export_state_native(self, box=0, state_out=None, owner_out=None):
        """Storage-format state (lb_export_state_native): state is a uint8
        array of native_bytes(box); state_out / owner_out: optional
        C-contiguous uint8 / int32 arrays to fill (e.g. pinned host memory)."""
        N, nb = self.n_nodes[box], self.native_bytes(box)
        if state_out is not None:
            if state_out.dtype != np.uint8 or state_out.size != nb or not state_out.flags.c_contiguous:
                raise ValueError("state_out must be a C-contiguous uint8 array of native_bytes() bytes")
            sa = state_out
        else:
            sa = np.zeros(nb, np.uint8)
        if owner_out is not None:
            if owner_out.dtype != np.int32 or owner_out.size != N or not owner_out.flags.c_contiguous:
                raise ValueError("owner_out must be a C-contiguous int32 array of N values")
            owner = owner_out
        else:
            owner = np.zeros(N, np.int32)
        parts = np.zeros((max(self.n_particles[box], 1), 9))
        meta = np.zeros(NATIVE_META)
        _ck(load_library().lb_export_state_native(self._h, box, sa.ctypes.data_as(C.c_void_p), sa.size, _ip(owner),
                                                  _dp(parts), _dp(meta)), "lb_export_state_native")
        return dict(state=sa, owner=owner, particles=parts[: self.n_particles[box]], meta=meta)

    def import_state_native(self, box, st):
        sa = st["state"]
        if sa.dtype != np.uint8 or not sa.flags.c_contiguous:
            raise ValueError("state must be a C-contiguous uint8 array")
        owner = np.ascontiguousarray(st["owner"], np.int32)
        parts = np.ascontiguousarray(st["particles"], np.float64).reshape(-1, 9)
        if parts.shape[0] == 0:
            parts = np.zeros((1, 9))
        meta = np.ascontiguousarray(st["meta"], np.float64)
        if meta.size != NATIVE_META:
            raise ValueError("meta must hold %d values" % NATIVE_META)
        _ck(load_library().lb_import_state_native(self._h, box, sa.ctypes.data_as(C.c_void_p), sa.size, _ip(owner),
                                                  _dp(parts), _dp(meta)), "lb_import_state_native")

    def rho(self, box=0):
        r = np.zeros((2, self.n_nodes[box]))
        _ck(load_library().lb_export_rho(self._h, box, _dp(r)), "lb_export_rho")
        return r

    def phi(self, box=0):
        """Order parameter rho^r - rho^b (0 on solid nodes), shape (nz, ny, nx)."""
        nx, ny, nz = self.dims[box]
        out = np.zeros(nx * ny * nz)
        _ck(load_library().lb_export_phi(self._h, box, _dp(out), None, None), "lb_export_phi")
        return out.reshape(nz, ny, nx)

    def structure(self, box=0):
        """Domain size (L_x, L_y, L_z) and interface coverage of one box."""
        L = np.zeros(3)
        cov = C.c_double(0)
        _ck(load_library().lb_export_phi(self._h, box, None, _dp(L), C.byref(cov)), "lb_export_phi")
        return L, cov.value

    def set_axes(self, box, e):
        """Body axes [n_particles][3] of spheroids (unit vectors)."""
        ee = np.ascontiguousarray(e, np.float64).reshape(-1, 3)
        _ck(load_library().lb_set_axes(self._h, box, _dp(ee)), "lb_set_axes")

    def axes(self, box=0):
        e = np.zeros((max(self.n_particles[box], 1), 3))
        _ck(load_library().lb_get_axes(self._h, box, _dp(e)), "lb_get_axes")
        return e[: self.n_particles[box]]

    def set_colors(self, box, colors):
        c = np.ascontiguousarray(colors, np.float64)
        _ck(load_library().lb_set_particle_colors(self._h, box, _dp(c)), "lb_set_particle_colors")

    def particle_forces(self, box=0):
        npb = max(self.n_particles[box], 1)
        F = np.zeros((npb, 3))
        T = np.zeros((npb, 3))
        _ck(load_library().lb_particle_forces(self._h, box, _dp(F), _dp(T)), "lb_particle_forces")
        return F[: self.n_particles[box]], T[: self.n_particles[box]]

    # -- tuning and timing ------------------------------------------------------------
    def set_tiling(self, ty, cz, split=0):
        _ck(load_library().lb_set_tiling(self._h, int(ty), int(cz), int(split)), "lb_set_tiling")

    def set_profiling(self, on):
        _ck(load_library().lb_set_profiling(self._h, 1 if on else 0), "lb_set_profiling")

    PHASES = ("lists", "remap_detect", "cover_uncover", "shell", "fused", "couple", "md")

    def phase_times(self):
        """Milliseconds per phase of the steps the last kernel_time() covered."""
        ms = np.zeros(len(self.PHASES))
        _ck(load_library().lb_phase_times(self._h, _dp(ms), len(ms)), "lb_phase_times")
        return dict(zip(self.PHASES, ms))

    def kernel_time(self):
        ms = C.c_double(0)
        nf, nt = C.c_int64(0), C.c_int64(0)
        _ck(load_library().lb_kernel_time(self._h, C.byref(ms), C.byref(nf), C.byref(nt)), "lb_kernel_time")
        return ms.value, nf.value, nt.value
