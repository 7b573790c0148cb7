"""Seeded synthetic inputs for the projection workloads (numpy only; none of the solver's arithmetic).

Both the CUDA path and the oracle consume these arrays; this module computes no part of the method.
Random numbers come from numpy's counter-based Philox generator.

Workloads (droplet fields standing in for the paper's droplet cases, §4.1 and §4.6):

* ``random_velocity``   face velocities i.i.d. N(0, sigma) on interior faces; faces on the boundary of a
                        bounded axis are 0 (impermeable wall).
* ``droplet``           liquid indicator C = (1 - tanh((r - R) / (1.5 dx))) / 2 of a sphere of radius 0.15 L,
                        centre L/2 + U(-0.1, 0.1) L per axis, periodic minimum image on periodic axes;
                        mdot = 1; rho1 = 100, rho2 = 1 (density ratio 100, Table tbl:table_groups).
* ``swirl_velocity``    solid-body rotation about the z axis through the droplet centre (Omega = 2) plus
                        N(0, 0.1) noise on interior faces.
* ``pressure_history``  p^n and p^{n-1} for the variable-density step: a pressure jump of 0.1 across the
                        droplet interface (0.1 C) plus N(0, 0.01) noise, and p^{n-1} = 0.95 p^n.
* ``stretched_dz``      tanh-clustered z widths with maximum neighbour ratio 1.05 (bisection on the
                        clustering parameter).
* ``batch_sizes`` / ``serve_sizes``  instance grid sizes for the batched and served workloads.
"""
import math

import numpy as np

BASE_SEED = 20190701


def rng(seed):
    return np.random.Generator(np.random.Philox(int(seed)))


def face_shapes(n, bc):
    """Shapes ([z][y][x]) of the u, v, w face arrays for grid size n = (nx, ny, nz)."""
    nx, ny, nz = n
    ex = [int(b != "P") for b in bc]
    return ((nz, ny, nx + ex[0]), (nz, ny + ex[1], nx), (nz + ex[2], ny, nx))


def _zero_walls(a, axis_np, bounded):
    if bounded:
        idx = [slice(None)] * 3
        idx[axis_np] = 0
        a[tuple(idx)] = 0.0
        idx[axis_np] = -1
        a[tuple(idx)] = 0.0
    return a


def random_velocity(n, bc, seed, sigma=1.0):
    g = rng(seed)
    out = []
    for axis, shp in enumerate(face_shapes(n, bc)):
        a = sigma * g.standard_normal(shp)
        out.append(_zero_walls(a, 2 - axis, bc[axis] != "P"))
    return tuple(out)


def uniform_dz(nz, L=1.0):
    return np.full(int(nz), L / nz)


def stretched_dz(nz, ratio=1.05, L=1.0):
    """Face positions z_k = (L/2)(1 + tanh(a (2k/nz - 1)) / tanh a), k = 0..nz; a chosen so that the largest
    ratio of neighbouring widths is ``ratio`` (clustered at both walls)."""
    k = np.arange(nz + 1)
    if nz < 3:
        return uniform_dz(nz, L)

    def widths(a):
        z = 0.5 * L * (1.0 + np.tanh(a * (2.0 * k / nz - 1.0)) / math.tanh(a))
        return np.diff(z)

    def max_ratio(a):
        w = widths(a)
        r = w[1:] / w[:-1]
        return float(np.max(np.maximum(r, 1.0 / r)))

    lo, hi = 1e-6, 8.0
    if max_ratio(hi) < ratio:
        return widths(hi)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if max_ratio(mid) < ratio:
            lo = mid
        else:
            hi = mid
    return widths(lo)


def droplet(n, bc, seed, L=1.0, radius=0.15, width_cells=1.5, dz=None):
    """Liquid indicator C at cell centres of an [0, L]^3 box (z widths ``dz`` if given) and its centre."""
    nx, ny, nz = n
    g = rng(seed)
    centre = L / 2 + g.uniform(-0.1, 0.1, size=3) * L
    dx = L / nx
    xc = (np.arange(nx) + 0.5) * dx
    yc = (np.arange(ny) + 0.5) * (L / ny)
    if dz is None:
        dz = uniform_dz(nz, L)
    zf = np.concatenate([[0.0], np.cumsum(dz)])
    zc = 0.5 * (zf[:-1] + zf[1:])
    d = []
    for axis, c in enumerate((xc, yc, zc)):
        r = c - centre[axis]
        if bc[axis] == "P":
            r = r - L * np.round(r / L)
        d.append(r)
    r = np.sqrt(d[2][:, None, None] ** 2 + d[1][None, :, None] ** 2 + d[0][None, None, :] ** 2)
    C = 0.5 * (1.0 - np.tanh((r - radius * L) / (width_cells * dx)))
    return C, centre


def swirl_velocity(n, bc, centre, seed, omega=2.0, noise=0.1, L=1.0):
    """u = -Omega (y - yc), v = Omega (x - xc), w = 0 on faces, plus N(0, noise) on interior faces."""
    nx, ny, nz = n
    g = rng(seed)
    su, sv, sw = face_shapes(n, bc)
    yc = (np.arange(ny) + 0.5) * (L / ny)
    xc = (np.arange(nx) + 0.5) * (L / nx)
    u = np.broadcast_to(-omega * (yc - centre[1])[None, :, None], su).copy()
    v = np.broadcast_to(omega * (xc - centre[0])[None, None, :], sv).copy()
    w = np.zeros(sw)
    out = []
    for axis, a in enumerate((u, v, w)):
        a = a + noise * g.standard_normal(a.shape)
        out.append(_zero_walls(a, 2 - axis, bc[axis] != "P"))
    return tuple(out)


def config_small(seed_offset=0):
    """32^3, periodic x, y, Neumann z, N(0,1) velocity; returns a dict of host arrays and grid parameters."""
    n = (32, 32, 32)
    bc = ("P", "P", "NN")
    u, v, w = random_velocity(n, bc, BASE_SEED + 1 + seed_offset)
    return dict(n=n, bc=bc, dx=1.0 / 32, dy=1.0 / 32, dz=uniform_dz(32), u=u, v=v, w=w, dt_over_rho0=1.0)


def config_droplet(N=128, seed_offset=0):
    """N^3 droplet step: swirl velocity, spherical indicator, mdot = 1, rho1 = 100, rho2 = 1."""
    n = (N, N, N)
    bc = ("P", "P", "NN")
    C, centre = droplet(n, bc, BASE_SEED + 2 + seed_offset)
    u, v, w = swirl_velocity(n, bc, centre, BASE_SEED + 102 + seed_offset)
    mdot = np.ones(C.shape)
    return dict(n=n, bc=bc, dx=1.0 / N, dy=1.0 / N, dz=uniform_dz(N), u=u, v=v, w=w, C=C, mdot=mdot,
                rho1=100.0, rho2=1.0, dt_over_rho0=1.0)


def pressure_history(C, seed, jump=0.1, noise=0.01):
    """(p^n, p^{n-1}) at cell centres: jump * C plus N(0, noise), and 0.95 times that."""
    pn = jump * np.asarray(C, dtype=np.float64) + noise * rng(seed).standard_normal(np.shape(C))
    return pn, 0.95 * pn


def batch_sizes(count=64, seed=BASE_SEED + 4, choices=(32, 48, 64, 96, 128, 160)):
    g = rng(seed)
    return [tuple(int(x) for x in g.choice(choices, size=3)) for _ in range(count)]


def serve_sizes(count, seed=BASE_SEED + 5, lo=48, hi=256):
    g = rng(seed)
    return [tuple(int(round(math.exp(x))) for x in g.uniform(math.log(lo), math.log(hi), size=3))
            for _ in range(count)]
