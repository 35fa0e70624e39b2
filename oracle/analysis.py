"""Observables of the oracle state (test infrastructure).

domain_size: Eq. eq:domsize.  L_i = 2 pi / sqrt(<k_i^2>), where <k_i^2> is
the S(k)-weighted mean of k_i^2, S(k) = |phi'_k|^2 / N and phi' = phi - <phi>.
Wave numbers k_i = 2 pi n_i / L_i with n_i in [-L_i/2, L_i/2 - 1].

contact_angle: Eq. eqn_contactangle_calculation.  cos(theta) = dh / R with
dh the distance along z from the particle centre to the interface, located
by linear interpolation of the phi = 0 crossing.

coverage: fraction of particles whose fluid neighbour nodes carry both signs
of phi (the paper names interface coverage but does not define it).  Parity
unpinned: the definition is a reading; a brute-force test pins only the code
against that reading, not the reading against the paper.
"""
import numpy as np


def domain_size(phi):
    """phi: array (nz, ny, nx).  Returns (L_x, L_y, L_z)."""
    phi = np.asarray(phi, dtype=np.float64)
    nz, ny, nx = phi.shape
    fluct = phi - phi.mean()
    S = np.abs(np.fft.fftn(fluct)) ** 2 / phi.size
    out = []
    for axis, n in ((2, nx), (1, ny), (0, nz)):
        k = 2.0 * np.pi * np.fft.fftfreq(n)  # same set as n_i in [-n/2, n/2-1] for even n
        shape = [1, 1, 1]
        shape[axis] = n
        k2 = (k ** 2).reshape(shape)
        tot = S.sum()
        m2 = (k2 * S).sum() / tot
        # a field uniform along this axis has no spectrum there: L = inf
        with np.errstate(divide="ignore"):
            out.append(2.0 * np.pi / np.sqrt(m2))
    return tuple(out)


def interface_height(phi_column):
    """Linear interpolation of the first + -> - (or - -> +) crossing of phi
    along a 1D column; returns the fractional index or None."""
    col = np.asarray(phi_column, dtype=np.float64)
    for k in range(len(col) - 1):
        a, b = col[k], col[k + 1]
        if a == 0.0:
            return float(k)
        if a * b < 0.0:
            return k + a / (a - b)
    return None


def contact_angle(dh, radius):
    """theta in degrees from cos(theta) = dh / R."""
    c = np.clip(dh / radius, -1.0, 1.0)
    return float(np.degrees(np.arccos(c)))


def coverage(phi, owner, n_particles):
    """phi, owner: arrays (nz, ny, nx); owner -1 fluid, p >= 0 particle p.
    A particle counts as covering the interface when the fluid nodes that
    are D3Q19 neighbours of its solid nodes include phi > 0 and phi < 0."""
    phi = np.asarray(phi, dtype=np.float64)
    owner = np.asarray(owner)
    if n_particles == 0:
        return 0.0
    pos = np.zeros(n_particles, bool)
    neg = np.zeros(n_particles, bool)
    offs = [(dx, dy, dz) for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1)
            if 0 < abs(dx) + abs(dy) + abs(dz) <= 2]
    solid = owner >= 0
    for dx, dy, dz in offs:
        # neighbour of each node along (dx, dy, dz)
        nb_owner = np.roll(owner, shift=(-dz, -dy, -dx), axis=(0, 1, 2))
        nb_phi = np.roll(phi, shift=(-dz, -dy, -dx), axis=(0, 1, 2))
        sel = solid & (nb_owner == -1)
        ps = owner[sel]
        vals = nb_phi[sel]
        pos[ps[vals > 0]] = True
        neg[ps[vals < 0]] = True
    return float(np.mean(pos & neg))
