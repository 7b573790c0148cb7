"""Exact direct solve of the MAC Poisson equation and the pressure projection (oracle; test infrastructure only).

The paper's flow solver reduces the pressure step to a constant-coefficient, second-order finite-difference
Poisson equation (§3.2, Eq. lap_p) and inverts it with a direct (FFT-based) solver; the Stefan potential of
§3.6 (Eq. ext_div) uses the same solver with the same boundary conditions.  A direct solver returns the exact
solution of the discrete linear system, so this module computes exactly that, by a route that shares nothing
with the GPU library:

1. If L is singular (no Dirichlet end on any axis) the volume-weighted mean of f is removed (the least-squares
   reading of an incompatible right-hand side) and reported as the compatibility defect.
2. The x and y 1-D operator matrices (symmetric, uniform spacing) are diagonalised by the textbook
   orthonormal Fourier / cosine / sine vectors at the cell centres (one dense basis matrix per axis), each
   eigenvalue taken as the Rayleigh quotient q^T A q of the stencil matrix A itself; f is transformed with
   the basis matrices (plain matrix products).
3. For every (x, y) eigenpair the z system (A_z + (lx + ly) I) p_hat = f_hat is solved: Thomas elimination
   for a bounded z axis, Sherman-Morrison around it for a periodic one, a bordered dense solve with the
   constraint sum(dz * p_hat) = 0 for the singular mode.
4. The inverse transform gives p.
5. The direct solve in FP64 loses about eps * cond(L) (about 1e-10 relative on a 512^3 grid with stretched z,
   mostly in the smoothest modes and, for a singular L, in the bordered solve of the mean mode), so the
   solution of the discrete system is then reached by one residual-correction step with the same solve,
   p += solve(f - fbar - L p), and the gauge of a singular L -- zero volume-weighted mean -- is imposed
   explicitly at the end.
"""
import numpy as np

from .mac import Grid, apply_laplacian, divergence, gradient, operator_matrix_1d


def _basis(n, bc):
    """Orthonormal eigenbasis (columns) of the uniform 1-D operator: the textbook Fourier, cosine and sine
    vectors at cell centres j + 1/2 for each boundary condition."""
    j = np.arange(n) + 0.5
    Q = np.empty((n, n))
    if bc == "P":
        Q[:, 0] = 1.0 / np.sqrt(n)
        col = 1
        for m in range(1, (n + 1) // 2):
            Q[:, col] = np.sqrt(2.0 / n) * np.cos(2 * np.pi * m * j / n)
            Q[:, col + 1] = np.sqrt(2.0 / n) * np.sin(2 * np.pi * m * j / n)
            col += 2
        if n % 2 == 0:
            Q[:, col] = np.cos(np.pi * (j - 0.5)) / np.sqrt(n)
        return Q
    for m in range(n):
        if bc == "NN":
            v = np.cos(np.pi * m * j / n)
        elif bc == "DD":
            v = np.sin(np.pi * (m + 1) * j / n)
        elif bc == "ND":
            v = np.cos(np.pi * (m + 0.5) * j / n)
        else:  # DN
            v = np.sin(np.pi * (m + 0.5) * j / n)
        Q[:, m] = v / np.linalg.norm(v)
    return Q


def _eig_axis(w, bc):
    """Eigenpairs of the x or y operator: the orthonormal basis above, with each eigenvalue taken as the
    Rayleigh quotient q^T A q of the stencil matrix itself.  (A numerical ``eigh`` loses about eps * cond in
    the low eigenvectors, which exceeds 1e-12 on long periodic axes.)"""
    A = operator_matrix_1d(w, bc)
    if not np.allclose(A, A.T, rtol=0, atol=1e-12 * np.abs(A).max()):
        raise ValueError("x/y operator must be symmetric (uniform spacing)")
    Q = _basis(A.shape[0], bc)
    lam = np.einsum("im,ij,jm->m", Q, A, Q)
    return lam, Q


def _bands(Az):
    n = Az.shape[0]
    a = np.zeros(n)   # sub-diagonal (coefficient of p_{k-1}) in row k
    c = np.zeros(n)   # super-diagonal (coefficient of p_{k+1}) in row k
    b = np.diag(Az).copy()
    for k in range(1, n):
        a[k] = Az[k, k - 1]
    for k in range(n - 1):
        c[k] = Az[k, k + 1]
    return a, b, c


def _thomas(a, b, c, lam, F):
    """Solve (tridiag(a, b, c) + diag(lam)) x = F for every mode at once; lam and F broadcast over modes."""
    n = F.shape[0]
    cp = np.empty_like(F)
    dp = np.empty_like(F)
    den = b[0] + lam
    cp[0] = c[0] / den
    dp[0] = F[0] / den
    for k in range(1, n):
        den = (b[k] + lam) - a[k] * cp[k - 1]
        cp[k] = c[k] / den
        dp[k] = (F[k] - a[k] * dp[k - 1]) / den
    x = np.empty_like(F)
    x[n - 1] = dp[n - 1]
    for k in range(n - 2, -1, -1):
        x[k] = dp[k] - cp[k] * x[k + 1]
    return x


def _solve_z(Az, bcz, lam, F):
    """Solve (A_z + lam I) x = F for all modes; ``lam`` has the mode shape, F is (nz, *mode shape)."""
    nz = Az.shape[0]
    if bcz != "P":
        a, b, c = _bands(Az)
        return _thomas(a, b[:, None, None], c, lam, F)
    if nz <= 2:
        # tiny cyclic systems: dense solve per mode
        M = F.reshape(nz, -1).T
        L = lam.reshape(-1)
        X = np.empty_like(M)
        for m in range(M.shape[0]):
            X[m] = np.linalg.solve(Az + L[m] * np.eye(nz), M[m])
        return X.T.reshape(F.shape)
    # cyclic tridiagonal: Sherman-Morrison with A = T + u v^T
    a, b, c = _bands(Az)
    alpha = Az[0, nz - 1]   # top-right corner
    beta = Az[nz - 1, 0]    # bottom-left corner
    gamma = -(b[0] + lam)   # per mode
    bb = np.broadcast_to(b[:, None, None] + lam[None], F.shape).copy()
    bb[0] = bb[0] - gamma
    bb[nz - 1] = bb[nz - 1] - alpha * beta / gamma
    zero = np.zeros_like(lam)
    y = _thomas(a, bb, c, zero, F)
    uvec = np.zeros_like(F)
    uvec[0] = gamma
    uvec[nz - 1] = beta
    z = _thomas(a, bb, c, zero, uvec)
    vy = y[0] + (alpha / gamma) * y[nz - 1]
    vz = z[0] + (alpha / gamma) * z[nz - 1]
    return y - (vy / (1.0 + vz))[None] * z


def _direct(grid, f):
    """One direct solve of L p = f (f compatible when L is singular): transforms, z systems, inverse."""
    lx, Qx = _eig_axis(grid.widths[0], grid.bc[0])
    ly, Qy = _eig_axis(grid.widths[1], grid.bc[1])
    wz = grid.widths[2]
    Az = operator_matrix_1d(wz, grid.bc[2])
    # forward transform: F[k, b, a] = sum_{j,i} Qy[j, b] Qx[i, a] f[k, j, i]
    F = np.matmul(f, Qx)                                  # over i
    F = np.matmul(Qy.T[None], F)                          # over j
    lam = ly[:, None] + lx[None, :]                       # (ny, nx) mode eigenvalue
    scale = np.abs(lx).max() + np.abs(ly).max() + 1.0
    sing = np.zeros(lam.shape, dtype=bool)
    if grid.bc[2] in ("P", "NN"):
        sing = np.abs(lam) <= 1e-10 * scale
    lam_safe = np.where(sing, -1.0, lam)
    P = _solve_z(Az, grid.bc[2], lam_safe, F)
    nz = Az.shape[0]
    for (bi, ai) in zip(*np.nonzero(sing)):
        # singular mode: A_z is singular with right null vector 1 and left null vector dz;
        # bordered system [[A_z, 1], [dz^T, 0]] picks the solution with sum(dz * p_hat) = 0
        B = np.zeros((nz + 1, nz + 1))
        B[:nz, :nz] = Az + lam[bi, ai] * np.eye(nz)
        B[:nz, nz] = 1.0
        B[nz, :nz] = wz
        rhs = np.concatenate([F[:, bi, ai], [0.0]])
        P[:, bi, ai] = np.linalg.solve(B, rhs)[:nz]
    # inverse transform
    p = np.matmul(Qy[None], P)
    p = np.matmul(p, Qx.T)
    return p


def poisson_solve(grid, f, corrections=1):
    """Return (p, info): the exact solution of L p = f - fbar in the gauge described in the module docstring.

    ``info`` holds ``compat_defect`` (the removed volume-weighted mean of f; 0 when L is regular).
    ``corrections``: residual-correction steps after the direct solve (module docstring, item 5).
    """
    f = np.asarray(f, dtype=np.float64)
    if f.shape != grid.shape:
        raise ValueError("f has shape %s, expected %s" % (f.shape, grid.shape))
    V = grid.cell_volumes()
    defect = 0.0
    if grid.singular():
        defect = float((f * V).sum() / V.sum())
        f = f - defect
    p = _direct(grid, f)
    for _ in range(corrections):
        p = p + _direct(grid, f - apply_laplacian(grid, p))
    if grid.singular():
        p = p - (p * V).sum() / V.sum()
    return p, {"compat_defect": defect}


def project(grid, u, v, w, src=None, dt_over_rho0=1.0):
    """Pressure projection (Eq. lap_p, constant-density part, and the correction step that follows it).

    f = (D u* - s) / (dt/rho0);  p solves L p = f - fbar;  u = u* - (dt/rho0) G p.
    Returns (u, v, w, p, info).
    """
    f = divergence(grid, u, v, w)
    if src is not None:
        f = f - np.asarray(src, dtype=np.float64)
    f = f / dt_over_rho0
    p, info = poisson_solve(grid, f)
    gu, gv, gw = gradient(grid, p)
    return (np.asarray(u) - dt_over_rho0 * gu, np.asarray(v) - dt_over_rho0 * gv,
            np.asarray(w) - dt_over_rho0 * gw, p, info)


def _face_mean(grid, q, axis):
    """Face values of a cell field: the mean of the two cells across each face (wrapped on a periodic axis);
    a bounded axis' end faces take their one adjacent cell."""
    from .mac import _NP_AXIS
    ax = _NP_AXIS[axis]
    n = grid.n[axis]
    q = np.asarray(q, dtype=np.float64)
    if grid.bc[axis] == "P":
        return 0.5 * (q + np.roll(q, 1, axis=ax))
    first = np.take(q, [0], axis=ax)
    last = np.take(q, [n - 1], axis=ax)
    inner = 0.5 * (np.take(q, np.arange(1, n), axis=ax) + np.take(q, np.arange(0, n - 1), axis=ax))
    return np.concatenate([first, inner, last], axis=ax)


def project_variable_density(grid, u, v, w, C, p_n, p_nm1, dt, dt_prev, rho1, rho2, src=None):
    """Pressure step with the variable-density pressure splitting of §3.2 (Eq. lap_p in full, and the velocity
    update that follows it), written term by term.

        p_hat   = (1 + dt/dt_prev) p^n - (dt/dt_prev) p^{n-1}
        rho     = rho1 C + rho2 (1 - C)                                   (Eq. material_prop, H ~ C)
        rho0    = min(rho1, rho2)
        L p / rho0 = D[(1/rho0 - 1/rho_f) G p_hat] + (D u* - s) / dt      (Eq. lap_p)
        u^{n+1} = u* - dt [ (1/rho0) G p + (1/rho_f - 1/rho0) G p_hat ]

    rho_f: rho on the faces, the mean of the two adjacent cells (a bounded axis' end face takes its cell) --
    a reading; the paper does not say how rho reaches the faces.  ``p_nm1`` None means p_hat = p^n.
    Returns (u, v, w, p, info).
    """
    rho0 = min(rho1, rho2)
    r = dt / dt_prev
    p_n = np.asarray(p_n, dtype=np.float64)
    p_hat = p_n if p_nm1 is None else (1.0 + r) * p_n - r * np.asarray(p_nm1, dtype=np.float64)
    rho = rho1 * np.asarray(C, dtype=np.float64) + rho2 * (1.0 - np.asarray(C, dtype=np.float64))
    gh = gradient(grid, p_hat)
    inv_rf = [1.0 / _face_mean(grid, rho, a) for a in range(3)]
    flux = [(1.0 / rho0 - inv_rf[a]) * gh[a] for a in range(3)]
    rhs = divergence(grid, *flux) + divergence(grid, u, v, w) / dt
    if src is not None:
        rhs = rhs - np.asarray(src, dtype=np.float64) / dt
    p, info = poisson_solve(grid, rho0 * rhs)
    gp = gradient(grid, p)
    vel = [np.asarray(x, dtype=np.float64) - dt * (gp[a] / rho0 + (inv_rf[a] - 1.0 / rho0) * gh[a])
           for a, x in enumerate((u, v, w))]
    return vel[0], vel[1], vel[2], p, info
