"""GB300 (sm_103a) implementation of the per-step hot path of the
two-component Shan-Chen D3Q19 lattice Boltzmann fluid with suspended
spheres of Jansen & Harting, arXiv:1004.4414.

The compute path is the C-ABI library built from csrc/ (include/lbpart.h);
binding.Simulation marshals arguments to it.  analysis holds host-side
observables (domain size, contact angle, coverage) of exported fields.
"""
from .binding import Simulation, make_params, load_library, LbError  # noqa: F401
