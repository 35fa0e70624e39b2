"""Seeded synthetic inputs shared by the CUDA path and the oracle in tests.

Holds none of the method's arithmetic: it only draws densities, particle
positions and velocities (numpy's PCG64 generator) in the shapes and value
ranges of the paper's runs -- a homogeneous mixture with node noise
(Sec. VI: "an identical amount of the two fluid species is distributed
randomly"), flat lamellae (Fig. 1 and the contact-angle set-up of Sec. V),
and non-overlapping spheres at random positions.

Arrays use the canonical node order n = x + nx*(y + ny*z); densities have
shape (2, N) for (red, blue); particles (np, 9) = X[3], U[3], omega[3].
"""
import numpy as np


def mixture(shape, rho_init=(0.7, 0.7), amp=0.01, seed=0):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    N = nx * ny * nz
    rho = np.empty((2, N))
    for c in range(2):
        rho[c] = rho_init[c] + amp * (2.0 * rng.random(N) - 1.0)
    return rho


def lamellae(shape, axis=2, rho_major=0.7, rho_minor=0.0, width=None, offset=0):
    """Red on [offset, offset+width) along `axis`, blue elsewhere."""
    nx, ny, nz = shape
    n = shape[axis]
    width = n // 2 if width is None else width
    coord = np.indices((nz, ny, nx))[2 - axis].reshape(-1)
    red = ((coord - offset) % n) < width
    rho = np.empty((2, nx * ny * nz))
    rho[0] = np.where(red, rho_major, rho_minor)
    rho[1] = np.where(red, rho_minor, rho_major)
    return rho


def layers(shape, period, rho_major=0.6, rho_minor=0.1, amp=0.01, seed=0):
    """Alternating red and blue layers along z, each period / 2 nodes thick
    (red first), with node noise U(-amp, amp) on both components."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    z = np.indices((nz, ny, nx))[0].reshape(-1)
    red = (z % period) < period // 2
    N = nx * ny * nz
    rho = np.empty((2, N))
    rho[0] = np.where(red, rho_major, rho_minor) + amp * (2.0 * rng.random(N) - 1.0)
    rho[1] = np.where(red, rho_minor, rho_major) + amp * (2.0 * rng.random(N) - 1.0)
    return rho


def spheres(shape, radius, n, seed=0, min_gap=0.0, vmax=0.0, wmax=0.0, max_tries=100000):
    """n centres with minimum-image distance >= 2R + min_gap, uniform
    velocities in [-vmax, vmax] and angular velocities in [-wmax, wmax]."""
    L = np.array(shape, dtype=np.float64)
    rng = np.random.default_rng(seed)
    X = []
    tries = 0
    while len(X) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place %d spheres" % n)
        c = rng.random(3) * L
        ok = True
        for o in X:
            d = c - o
            d -= L * np.round(d / L)
            if np.dot(d, d) < (2 * radius + min_gap) ** 2:
                ok = False
                break
        if ok:
            X.append(c)
    P = np.zeros((n, 9))
    if n:
        P[:, 0:3] = np.array(X)
        P[:, 3:6] = vmax * (2.0 * rng.random((n, 3)) - 1.0)
        P[:, 6:9] = wmax * (2.0 * rng.random((n, 3)) - 1.0)
    return P
