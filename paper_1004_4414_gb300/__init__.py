"""GB300 (sm_103a) implementation of the per-step hot path of the
two-component Shan-Chen D3Q19 lattice Boltzmann fluid with suspended
spheres of Jansen & Harting, arXiv:1004.4414.

The compute path is the C-ABI library built from csrc/ (include/lbpart.h);
binding.Simulation marshals arguments to it.  The observables of the
paper's runs (mass, momentum, the domain size of Eq. eq:domsize, interface
coverage, the order parameter) are computed on the device by the library.
"""
from .binding import Simulation, make_params, load_library, LbError  # noqa: F401
