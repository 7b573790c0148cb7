"""MAC-grid finite-difference operators (oracle; test infrastructure only).

The paper's solver works on a Cartesian grid with a marker-and-cell arrangement: pressure and scalars at
cell centres, velocity components on the cell faces, second-order finite differences (§3, first
paragraph; §3.2).  Boundary conditions are homogeneous and per axis (§3.2, last paragraph of the flow
solver description: "several combinations of homogeneous pressure boundary conditions").

Conventions (readings where the paper is silent; each is listed in the design notes):

* Arrays are C-ordered ``[k][j][i]`` (z slowest, x fastest).
* Axis widths: x and y uniform (``dx``, ``dy``); z has per-cell widths ``dz[k]`` (uniform in the paper,
  stretched in the 512^3 workload).
* Boundary condition per axis, one of ``P`` (periodic), ``NN``, ``DD``, ``ND``, ``DN`` (first letter = low
  end, second = high end).  ``N``: zero normal gradient at the boundary face (ghost value = p).
  ``D``: p = 0 at the boundary face (ghost value = -p, mirrored across the face).
* Face arrays: index ``i`` is the LOW face of cell ``i`` (x = i*dx).  A periodic axis stores ``n`` faces
  (face n is face 0); a bounded axis stores ``n + 1`` faces, both boundary faces included.
"""
import numpy as np

BCS = ("P", "NN", "DD", "ND", "DN")


class Grid:
    """Grid geometry: sizes, spacings and per-axis boundary conditions."""

    def __init__(self, nx, ny, nz, dx, dy, dz, bc):
        self.n = (int(nx), int(ny), int(nz))
        dz = np.broadcast_to(np.asarray(dz, dtype=np.float64), (int(nz),)).copy()
        self.widths = (np.full(int(nx), float(dx)), np.full(int(ny), float(dy)), dz)
        self.bc = tuple(bc)
        for b in self.bc:
            if b not in BCS:
                raise ValueError("unknown boundary condition %r" % (b,))
        if min(self.n) < 1 or np.any(dz <= 0) or dx <= 0 or dy <= 0:
            raise ValueError("bad grid")

    @property
    def shape(self):
        """Cell array shape, C order [z][y][x]."""
        return (self.n[2], self.n[1], self.n[0])

    def cell_volumes(self):
        wx, wy, wz = self.widths
        return wz[:, None, None] * wy[None, :, None] * wx[None, None, :]

    def singular(self):
        """True when L has the constants in its null space (no axis has a Dirichlet end)."""
        return all(b in ("P", "NN") for b in self.bc)


# numpy axis of each physical axis in a [z][y][x] array
_NP_AXIS = (2, 1, 0)


def face_shape(grid, axis):
    """Shape of the face array normal to ``axis`` (0 = x, 1 = y, 2 = z)."""
    s = list(grid.shape)
    if grid.bc[axis] != "P":
        s[_NP_AXIS[axis]] += 1
    return tuple(s)


def _bshape(axis, arr):
    """Reshape a 1-D per-axis array so it broadcasts along ``axis`` of a [z][y][x] array."""
    shp = [1, 1, 1]
    shp[_NP_AXIS[axis]] = arr.shape[0]
    return arr.reshape(shp)


def _ghost_distances(w, bc):
    """Centre-to-ghost-centre distance at the low and high ends of an axis.

    Periodic: the ghost is the wrapped cell, (w[n-1] + w[0]) / 2 away.  Bounded: the ghost is the mirror
    image of the end cell across the boundary face, one cell width away.
    """
    if bc == "P":
        h = 0.5 * (w[-1] + w[0])
        return h, h
    return w[0], w[-1]


def _face_spacing(w, bc):
    """Distance between the two cell centres on either side of each stored face."""
    n = w.shape[0]
    h = np.empty(n if bc == "P" else n + 1)
    h[1:n] = 0.5 * (w[:-1] + w[1:])
    lo, hi = _ghost_distances(w, bc)
    h[0] = lo
    if bc != "P":
        h[n] = hi
    return h


def gradient(grid, p):
    """Face-normal gradient G p on the three face arrays (the correction step after Eq. lap_p).

    Interior faces: (p_i - p_{i-1}) / h.  Boundary faces of a bounded axis: 0 at an N end; at a D end the
    ghost value -p gives 2 p_0 / w_0 (low) and -2 p_{n-1} / w_{n-1} (high).
    """
    p = np.asarray(p, dtype=np.float64)
    out = []
    for axis in range(3):
        ax = _NP_AXIS[axis]
        n = grid.n[axis]
        w = grid.widths[axis]
        bc = grid.bc[axis]
        h = _face_spacing(w, bc)
        g = np.zeros(face_shape(grid, axis))
        sl = [slice(None)] * 3
        # interior faces 1..n-1
        sl_f = list(sl); sl_f[ax] = slice(1, n)
        sl_a = list(sl); sl_a[ax] = slice(1, n)
        sl_b = list(sl); sl_b[ax] = slice(0, n - 1)
        hb = _bshape(axis, h[1:n])
        g[tuple(sl_f)] = (p[tuple(sl_a)] - p[tuple(sl_b)]) / hb
        s0 = list(sl); s0[ax] = 0
        sl_last = list(sl); sl_last[ax] = n - 1
        if bc == "P":
            g[tuple(s0)] = (p[tuple(s0)] - p[tuple(sl_last)]) / h[0]
        else:
            if bc[0] == "D":
                g[tuple(s0)] = 2.0 * p[tuple(s0)] / w[0]
            sn = list(sl); sn[ax] = n
            if bc[1] == "D":
                g[tuple(sn)] = -2.0 * p[tuple(sl_last)] / w[n - 1]
        out.append(g)
    return tuple(out)


def divergence(grid, u, v, w):
    """Cell-centred divergence D u = sum over axes of (F_{i+1} - F_i) / w_i (Eq. mass, discretised)."""
    d = np.zeros(grid.shape)
    for axis, F in enumerate((u, v, w)):
        F = np.asarray(F, dtype=np.float64)
        if F.shape != face_shape(grid, axis):
            raise ValueError("face array %d has shape %s, expected %s" % (axis, F.shape, face_shape(grid, axis)))
        ax = _NP_AXIS[axis]
        n = grid.n[axis]
        hi = np.roll(F, -1, axis=ax) if grid.bc[axis] == "P" else np.take(F, np.arange(1, n + 1), axis=ax)
        lo = F if grid.bc[axis] == "P" else np.take(F, np.arange(0, n), axis=ax)
        d += (hi - lo) / _bshape(axis, grid.widths[axis])
    return d


def apply_laplacian(grid, p):
    """L p by the 7-point ghost-cell stencil, written independently of ``divergence`` and ``gradient``.

    Per axis: [(p_{i+1} - p_i)/h_{i+1/2} - (p_i - p_{i-1})/h_{i-1/2}] / w_i with ghost cells beyond the
    ends (wrapped for P, copied for N, negated for D).
    """
    p = np.asarray(p, dtype=np.float64)
    out = np.zeros_like(p)
    for axis in range(3):
        ax = _NP_AXIS[axis]
        n = grid.n[axis]
        w = grid.widths[axis]
        bc = grid.bc[axis]
        first = np.take(p, [0], axis=ax)
        last = np.take(p, [n - 1], axis=ax)
        if bc == "P":
            g_lo, g_hi = last, first
        else:
            g_lo = first if bc[0] == "N" else -first
            g_hi = last if bc[1] == "N" else -last
        padded = np.concatenate([g_lo, p, g_hi], axis=ax)
        # centre distances between consecutive entries of the padded line (n + 1 of them)
        lo_d, hi_d = _ghost_distances(w, bc)
        hc = np.concatenate([[lo_d], 0.5 * (w[:-1] + w[1:]), [hi_d]])
        up = np.take(padded, np.arange(2, n + 2), axis=ax)
        mid = np.take(padded, np.arange(1, n + 1), axis=ax)
        dn = np.take(padded, np.arange(0, n), axis=ax)
        flux_hi = (up - mid) / _bshape(axis, hc[1:])
        flux_lo = (mid - dn) / _bshape(axis, hc[:-1])
        out += (flux_hi - flux_lo) / _bshape(axis, w)
    return out


def operator_matrix_1d(w, bc):
    """Dense n x n matrix of the 1-D second-difference operator with the ghost rules of ``apply_laplacian``.

    Row i holds the weights of p_{i-1}, p_i, p_{i+1}; ghost weights fold into the diagonal (N: +, D: -) or
    wrap to the far end (P).
    """
    w = np.asarray(w, dtype=np.float64)
    n = w.shape[0]
    A = np.zeros((n, n))
    lo_d, hi_d = _ghost_distances(w, bc)
    for i in range(n):
        h_lo = lo_d if i == 0 else 0.5 * (w[i - 1] + w[i])
        h_hi = hi_d if i == n - 1 else 0.5 * (w[i] + w[i + 1])
        a = 1.0 / (w[i] * h_lo)   # weight of the lower neighbour
        c = 1.0 / (w[i] * h_hi)   # weight of the upper neighbour
        A[i, i] -= a + c
        if i > 0:
            A[i, i - 1] += a
        elif bc == "P":
            A[i, n - 1] += a
        else:
            A[i, i] += a if bc[0] == "N" else -a
        if i < n - 1:
            A[i, i + 1] += c
        elif bc == "P":
            A[i, 0] += c
        else:
            A[i, i] += c if bc[1] == "N" else -c
    return A
