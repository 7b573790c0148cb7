"""Stefan-potential solve, divergence-free liquid-velocity extension and interface velocity (oracle).

TEST INFRASTRUCTURE ONLY.  Follows §3.6 of the paper:

* regularised delta |grad C| (§3.2: discretised with Youngs' method; §3.6, Eq. ext_div);
* Stefan potential: lap(phi) = mdot (1/rho2 - 1/rho1) |grad C|, same solver and boundary conditions as the
  pressure (Eq. ext_div and the boundary-condition remark that follows Eq. ext_div_var_coeff);
* extended liquid velocity u1e = u - grad(phi)  (Eq. jump_subtr);
* interface velocity uG = u1e - (mdot / rho1) n  (Eq. int_vel).

Readings (the paper leaves these open):

* ``mode=0`` (default): cell-centred central differences, (C_{i+1} - C_{i-1}) / (h_{i-1/2} + h_{i+1/2}).
  ``mode=1``: Youngs' corner-gradient average: face differences averaged over the 2x2 cells around each of
  the 8 corners of the cell, then averaged over those corners.  Ghost cells copy C at bounded ends (C has a
  zero normal gradient at walls) and wrap at periodic ends.
* Normal sign: n points into the gas (Eq. rankine), and C = 1 in the liquid, so n = -grad C / |grad C|.
* n = 0 where min(C, 1 - C) < clip (default 1e-8, the cut-off used for the static-droplet figure of §4.1)
  or where |grad C| = 0.
* Face values of mdot and n: arithmetic mean of the two adjacent cells; a boundary face of a bounded axis
  takes the value of its one adjacent cell.
"""
import numpy as np

from .mac import Grid, face_shape, gradient, _NP_AXIS, _bshape, _ghost_distances
from .poisson import poisson_solve


def _pad_copy(grid, q, axis):
    """q with one ghost layer at each end of ``axis``: wrapped (P) or copied (bounded)."""
    ax = _NP_AXIS[axis]
    n = grid.n[axis]
    first = np.take(q, [0], axis=ax)
    last = np.take(q, [n - 1], axis=ax)
    if grid.bc[axis] == "P":
        return np.concatenate([last, q, first], axis=ax)
    return np.concatenate([first, q, last], axis=ax)


def _centre_spacings(grid, axis):
    """Centre distances between consecutive entries of a ghost-padded line (n + 1 values)."""
    w = grid.widths[axis]
    lo, hi = _ghost_distances(w, grid.bc[axis])
    return np.concatenate([[lo], 0.5 * (w[:-1] + w[1:]), [hi]])


def grad_c(grid, C, mode=0):
    """Cell-centred gradient of the volume fraction C (three arrays, cell shape)."""
    C = np.asarray(C, dtype=np.float64)
    out = []
    for axis in range(3):
        ax = _NP_AXIS[axis]
        n = grid.n[axis]
        Cp = _pad_copy(grid, C, axis)
        h = _centre_spacings(grid, axis)
        if mode == 0:
            up = np.take(Cp, np.arange(2, n + 2), axis=ax)
            dn = np.take(Cp, np.arange(0, n), axis=ax)
            out.append((up - dn) / _bshape(axis, h[:-1] + h[1:]))
            continue
        # Youngs: face differences at the n + 1 faces along ``axis``
        Dface = (np.take(Cp, np.arange(1, n + 2), axis=ax) - np.take(Cp, np.arange(0, n + 1), axis=ax)) \
            / _bshape(axis, h)
        # transverse (1, 2, 1) / 4 smoothing over both other axes == averaging over the 4 corners
        for t in range(3):
            if t == axis:
                continue
            tax = _NP_AXIS[t]
            m = grid.n[t]
            Dp = _pad_copy(grid, Dface, t)
            Dface = 0.25 * (np.take(Dp, np.arange(0, m), axis=tax) + 2.0 * np.take(Dp, np.arange(1, m + 1), axis=tax)
                            + np.take(Dp, np.arange(2, m + 2), axis=tax))
        out.append(0.5 * (np.take(Dface, np.arange(0, n), axis=ax) + np.take(Dface, np.arange(1, n + 1), axis=ax)))
    return tuple(out)


def delta_and_normal(grid, C, mode=0, clip=1e-8):
    """Return (|grad C|, (n_x, n_y, n_z)) at cell centres with n = -grad C / |grad C| (0 where clipped)."""
    C = np.asarray(C, dtype=np.float64)
    g = grad_c(grid, C, mode)
    mag = np.sqrt(g[0] ** 2 + g[1] ** 2 + g[2] ** 2)
    ok = (np.minimum(C, 1.0 - C) >= clip) & (mag > 0)
    safe = np.where(ok, mag, 1.0)
    n = tuple(np.where(ok, -gi / safe, 0.0) for gi in g)
    return mag, n


def stefan_source(grid, C, mdot, rho1, rho2, mode=0):
    """s = mdot (1/rho2 - 1/rho1) |grad C| (right-hand side of Eq. ext_div and source term of Eq. lap_p)."""
    mag, _ = delta_and_normal(grid, C, mode)
    return np.asarray(mdot, dtype=np.float64) * (1.0 / rho2 - 1.0 / rho1) * mag


def face_average(grid, q, axis):
    """Face values of a cell field: mean of the two neighbours; a bounded axis' end faces copy their cell."""
    ax = _NP_AXIS[axis]
    n = grid.n[axis]
    qp = _pad_copy(grid, q, axis)
    lo = np.take(qp, np.arange(0, n + 1), axis=ax)
    hi = np.take(qp, np.arange(1, n + 2), axis=ax)
    f = 0.5 * (lo + hi)
    if grid.bc[axis] == "P":
        f = np.take(f, np.arange(0, n), axis=ax)
    return f


def extend_liquid_velocity(grid, u, v, w, C, mdot, rho1, rho2, mode=0, clip=1e-8):
    """Divergence-free liquid-velocity extension and interface velocity (§3.6).

    Returns (u1e, v1e, w1e, uG, vG, wG, phi, info).
    """
    s = stefan_source(grid, C, mdot, rho1, rho2, mode)
    phi, info = poisson_solve(grid, s)
    g = gradient(grid, phi)
    ue = tuple(np.asarray(q, dtype=np.float64) - gq for q, gq in zip((u, v, w), g))
    _, n = delta_and_normal(grid, C, mode, clip)
    mdot = np.broadcast_to(np.asarray(mdot, dtype=np.float64), grid.shape)
    ug = tuple(ue[a] - face_average(grid, mdot, a) / rho1 * face_average(grid, n[a], a) for a in range(3))
    return ue + ug + (phi, info)


def extend_vapour_velocity(grid, u, v, w, C, mdot, rho1, rho2, mode=0, clip=1e-8):
    """The boiling variant (Appendix A): the interface velocity from a divergence-free extension of the vapour
    (phase 2) velocity instead of the liquid's.

    Reading: exchanging the phases in §3.6 (C -> 1 - C, n -> -n, mdot -> -mdot, rho1 <-> rho2) leaves the
    Stefan source of Eq. ext_div, hence phi and u - grad(phi) of Eq. jump_subtr, unchanged; Eq. rankine
    written for the vapour side then gives uG = u2e - (mdot / rho2) n.  Returns (u2e, v2e, w2e, uG, vG, wG, phi,
    info).
    """
    s = stefan_source(grid, C, mdot, rho1, rho2, mode)
    phi, info = poisson_solve(grid, s)
    g = gradient(grid, phi)
    ue = tuple(np.asarray(q, dtype=np.float64) - gq for q, gq in zip((u, v, w), g))
    _, n = delta_and_normal(grid, C, mode, clip)
    mdot = np.broadcast_to(np.asarray(mdot, dtype=np.float64), grid.shape)
    ug = tuple(ue[a] - face_average(grid, mdot, a) / rho2 * face_average(grid, n[a], a) for a in range(3))
    return ue + ug + (phi, info)
