"""Volume-of-fluid update with the interface velocity (oracle; test infrastructure only).

TEST INFRASTRUCTURE ONLY.  Follows §3.1 of the paper: C is advected by the interface velocity uG (not the
one-fluid velocity) with a directional split, each one-dimensional step implicit in its own result (Eq.
fluxes), then the correction of Eq. final_corr_1 extended by the implicit volume-deflation term of Eq.
final_corr_2:

    C*   (1 - dt/dx (uG_{i+1/2} - uG_{i-1/2})) = C^n  - (f_{i+1/2} - f_{i-1/2}) / dx      (x, fluxes of C^n)
    C**  (1 - dt/dy (vG_{j+1/2} - vG_{j-1/2})) = C*   - (g_{j+1/2} - g_{j-1/2}) / dy      (y, fluxes of C*)
    C*** (1 - dt/dz_k (wG_{k+1/2} - wG_{k-1/2})) = C** - (h_{k+1/2} - h_{k-1/2}) / dz_k   (z, fluxes of C**)
    F    = C* du/dx + C** dv/dy + C*** dw/dz      (the face differences of uG above)
    C^{n+1} (1 - dt div(uG)) = C*** - dt F.

Reading: the paper takes its numerical fluxes f, g, h from the MTHINC reconstruction of its reference [ii2012],
which it does not restate; here they are first-order upwind fluxes, f_{i+1/2} = dt uG_{i+1/2} C_upwind (the
cell the face velocity comes from; on a bounded axis the outside cell is a copy of the boundary cell).
Only the split-update skeleton and its volume bookkeeping are the paper's.
"""
import numpy as np

from .mac import _NP_AXIS, _bshape


def _upwind_flux(grid, q, vel, axis, dt):
    """dt * vel * q_upwind on the faces of `axis` (the face array's own shape)."""
    ax = _NP_AXIS[axis]
    n = grid.n[axis]
    if grid.bc[axis] == "P":
        lo = np.roll(q, 1, axis=ax)  # cell i-1 across face i
        hi = q                       # cell i
    else:
        first = np.take(q, [0], axis=ax)
        last = np.take(q, [n - 1], axis=ax)
        lo = np.concatenate([first, q], axis=ax)   # faces 0..n: the cell below (a copy at face 0)
        hi = np.concatenate([q, last], axis=ax)    # the cell above (a copy at face n)
    return dt * vel * np.where(vel >= 0, lo, hi)


def _face_difference(grid, F, axis):
    """F_{i+1/2} - F_{i-1/2} per cell along `axis` (faces stored low face first)."""
    ax = _NP_AXIS[axis]
    n = grid.n[axis]
    if grid.bc[axis] == "P":
        return np.roll(F, -1, axis=ax) - F
    return np.take(F, np.arange(1, n + 1), axis=ax) - np.take(F, np.arange(0, n), axis=ax)


def vof_update(grid, C, uG, vG, wG, dt):
    """One split VoF step (Eqs. fluxes, final_corr_1, final_corr_2) with upwind fluxes.  Returns C^{n+1}."""
    q = np.asarray(C, dtype=np.float64)
    vel = [np.asarray(x, dtype=np.float64) for x in (uG, vG, wG)]
    stages = []
    dv = []
    for axis in range(3):
        w = _bshape(axis, np.asarray(grid.widths[axis], dtype=np.float64))
        flux = _upwind_flux(grid, q, vel[axis], axis, dt)
        du = _face_difference(grid, vel[axis], axis) / w
        q = (q - _face_difference(grid, flux, axis) / w) / (1.0 - dt * du)
        stages.append(q)
        dv.append(du)
    F = stages[0] * dv[0] + stages[1] * dv[1] + stages[2] * dv[2]
    return (stages[2] - dt * F) / (1.0 - dt * (dv[0] + dv[1] + dv[2]))
