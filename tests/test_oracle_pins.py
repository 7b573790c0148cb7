"""Pins of the CPU oracle against facts fixed by the paper and by the mathematics (no GPU).

* closed-form discrete eigenfunctions of the MAC Laplacian per boundary condition (cos / sin bases);
* brute force: the full 3-D matrix of the stencil, solved by dense LU (bordered for the singular case);
* Green's identity, D G = L consistency, the 1-D matrices vs the 3-D stencil;
* projection invariants: zero-mean gauge, machine-epsilon divergence, idempotence, discrete Pythagoras,
  linearity, translation equivariance, x <-> y symmetry;
* the extension of §3.6: exact decomposition u = u_df + grad(psi), the static-droplet case of §4.1
  (u1e = 0, uG = -(mdot/rho1) n), divergence-free u1e (Eq. jump_subtr), planar-interface normals;
* Youngs' corner-average gradient (§3.2) against closed forms on quadratic and periodic-wave fields and a
  corner-by-corner restatement; face values of Eq. int_vel against linear fields at the face position.
"""
import itertools
import json
import math
import os
import zlib

import numpy as np
import pytest

import oracle
from oracle import Grid
from paper_1907_00890_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
XY_BCS = ("P", "NN", "DD")
Z_BCS = ("P", "NN", "DD", "ND", "DN")


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


# ---- closed forms ---------------------------------------------------------------------------------------

def basis_1d(bc, n, m):
    """Closed-form eigenvector (cell centres j + 1/2) and eigenvalue times h^2 of the 1-D operator."""
    j = np.arange(n) + 0.5
    if bc == "P":
        return np.cos(2 * math.pi * m * j / n), -4 * math.sin(math.pi * m / n) ** 2
    if bc == "NN":
        return np.cos(math.pi * m * j / n), -4 * math.sin(math.pi * m / (2 * n)) ** 2
    if bc == "DD":
        return np.sin(math.pi * (m + 1) * j / n), -4 * math.sin(math.pi * (m + 1) / (2 * n)) ** 2
    if bc == "ND":
        return np.cos(math.pi * (m + 0.5) * j / n), -4 * math.sin(math.pi * (2 * m + 1) / (4 * n)) ** 2
    if bc == "DN":
        return np.sin(math.pi * (m + 0.5) * j / n), -4 * math.sin(math.pi * (2 * m + 1) / (4 * n)) ** 2
    raise ValueError(bc)


@pytest.mark.parametrize("bc", Z_BCS)
@pytest.mark.parametrize("n", [1, 2, 3, 7, 8, 16])
def test_1d_spectrum_closed_form(bc, n):
    h = 0.37
    A = oracle.operator_matrix_1d(np.full(n, h), bc)
    ev = np.sort(np.linalg.eigvals(A).real)
    closed = np.sort([basis_1d(bc, n, m)[1] / h ** 2 for m in range(n)])
    assert np.allclose(ev, closed, rtol=0, atol=1e-10 / h ** 2)
    for m in range(n):
        phi, lam = basis_1d(bc, n, m)
        assert np.allclose(A @ phi, lam / h ** 2 * phi, atol=1e-11 / h ** 2)


@pytest.mark.parametrize("bcx,bcy,bcz", list(itertools.product(XY_BCS, XY_BCS, Z_BCS)))
def test_closed_form_eigenfunction_recovered(bcx, bcy, bcz):
    n = (8, 6, 10)
    h = (0.125, 0.2, 0.1)
    g = Grid(*n, h[0], h[1], np.full(n[2], h[2]), (bcx, bcy, bcz))
    r = np.random.default_rng(zlib.crc32((bcx + bcy + bcz).encode()))
    f = np.zeros(g.shape)
    pstar = np.zeros(g.shape)
    for _ in range(3):
        ms = [int(r.integers(0, n[a])) for a in range(3)]
        if all(b in ("P", "NN") for b in (bcx, bcy, bcz)) and ms == [0, 0, 0]:
            ms[0] = 1
        parts = [basis_1d(b, n[a], ms[a]) for a, b in enumerate((bcx, bcy, bcz))]
        mode = parts[2][0][:, None, None] * parts[1][0][None, :, None] * parts[0][0][None, None, :]
        lam = sum(parts[a][1] / h[a] ** 2 for a in range(3))
        c = r.standard_normal()
        pstar += c * mode
        f += c * lam * mode
    assert np.allclose(oracle.apply_laplacian(g, pstar), f, atol=1e-10 * np.abs(f).max())
    p, info = oracle.poisson_solve(g, f)
    # non-constant eigenfunctions are orthogonal to constants, so the zero-mean gauge keeps p* itself
    assert rel(p, pstar) < 1e-12
    assert abs(info["compat_defect"]) < 1e-12 * np.abs(f).max()


# ---- brute force ----------------------------------------------------------------------------------------

def dense_operator(g):
    N = int(np.prod(g.shape))
    A = np.zeros((N, N))
    e = np.zeros(N)
    for c in range(N):
        e[:] = 0.0
        e[c] = 1.0
        A[:, c] = oracle.apply_laplacian(g, e.reshape(g.shape)).ravel()
    return A


def brute_solve(g, f):
    A = dense_operator(g)
    N = A.shape[0]
    V = g.cell_volumes().ravel()
    if g.singular():
        fbar = (f.ravel() * V).sum() / V.sum()
        B = np.zeros((N + 1, N + 1))
        B[:N, :N] = A
        B[:N, N] = 1.0
        B[N, :N] = V
        x = np.linalg.solve(B, np.concatenate([f.ravel() - fbar, [0.0]]))[:N]
    else:
        x = np.linalg.solve(A, f.ravel())
    return x.reshape(g.shape)


BRUTE_SIZES = [(8, 8, 8), (5, 3, 7), (1, 6, 8), (4, 4, 3), (3, 1, 2), (2, 2, 1)]


@pytest.mark.parametrize("bcx,bcy,bcz", list(itertools.product(XY_BCS, XY_BCS, Z_BCS)))
def test_brute_force_dense_lu(bcx, bcy, bcz):
    r = np.random.default_rng(7)
    for n in BRUTE_SIZES:
        dz = r.uniform(0.5, 1.5, n[2]) / n[2]
        g = Grid(*n, 1.0 / n[0], 0.7 / n[1], dz, (bcx, bcy, bcz))
        f = r.standard_normal(g.shape)
        p, _ = oracle.poisson_solve(g, f)
        pb = brute_solve(g, f)
        assert rel(p, pb) < 1e-11, (n, rel(p, pb))


# ---- operator identities --------------------------------------------------------------------------------

def face_weights(g, axis):
    """Face control volumes: area x centre distance; half a cell at a D boundary face, 0 at an N face."""
    w = g.widths[axis]
    n = g.n[axis]
    bc = g.bc[axis]
    area = g.cell_volumes() / oracle.mac._bshape(axis, w)
    area = np.take(area, [0], axis=oracle.mac._NP_AXIS[axis])
    h = np.zeros(n if bc == "P" else n + 1)
    h[1:n] = 0.5 * (w[:-1] + w[1:])
    if bc == "P":
        h[0] = 0.5 * (w[-1] + w[0])
    else:
        h[0] = 0.5 * w[0] if bc[0] == "D" else 0.0
        h[n] = 0.5 * w[-1] if bc[1] == "D" else 0.0
    return area * oracle.mac._bshape(axis, h)


@pytest.mark.parametrize("bcx,bcy,bcz", [("P", "P", "NN"), ("DD", "NN", "DN"), ("NN", "DD", "P"), ("P", "DD", "ND")])
def test_green_identity_and_dg(bcx, bcy, bcz):
    r = np.random.default_rng(3)
    n = (6, 5, 9)
    g = Grid(*n, 0.2, 0.3, r.uniform(0.3, 2.0, n[2]), (bcx, bcy, bcz))
    p = r.standard_normal(g.shape)
    q = r.standard_normal(g.shape)
    Lp = oracle.apply_laplacian(g, p)
    lhs = (g.cell_volumes() * q * Lp).sum()
    Gp = oracle.gradient(g, p)
    Gq = oracle.gradient(g, q)
    rhs = -sum((face_weights(g, a) * Gq[a] * Gp[a]).sum() for a in range(3))
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)
    assert np.allclose(oracle.divergence(g, *Gp), Lp, rtol=0, atol=1e-12 * np.abs(Lp).max())
    # the Kronecker sum of the 1-D matrices is the 3-D stencil
    Ax = oracle.operator_matrix_1d(g.widths[0], bcx)
    Ay = oracle.operator_matrix_1d(g.widths[1], bcy)
    Az = oracle.operator_matrix_1d(g.widths[2], bcz)
    K = np.einsum("ia,kji->kja", Ax.T, p) + np.einsum("jb,kji->kbi", Ay.T, p) + np.einsum("kc,kji->cji", Az.T, p)
    assert np.allclose(K, Lp, rtol=0, atol=1e-12 * np.abs(Lp).max())


# ---- projection invariants -----------------------------------------------------------------------------

def face_inner(g, a, b):
    return sum((face_weights(g, ax) * a[ax] * b[ax]).sum() for ax in range(3))


@pytest.mark.parametrize("bc", [("P", "P", "NN"), ("P", "P", "P"), ("NN", "DD", "DN"), ("DD", "DD", "DD")])
def test_projection_invariants(bc):
    n = (12, 10, 14)
    r = np.random.default_rng(11)
    dz = synth.stretched_dz(n[2]) if bc[2] != "P" else synth.uniform_dz(n[2])
    g = Grid(*n, 1.0 / n[0], 1.0 / n[1], dz, bc)
    u = synth.random_velocity(n, bc, 5)
    d0 = np.abs(oracle.divergence(g, *u)).max()
    s = 0.37
    u1, v1, w1, p, info = oracle.project(g, *u, src=None, dt_over_rho0=s)
    # machine-epsilon divergence and zero-mean gauge
    assert np.abs(oracle.divergence(g, u1, v1, w1)).max() < 1e-12 * d0
    if g.singular():
        assert abs((g.cell_volumes() * p).sum()) < 1e-13 * np.abs(p).max()
    # idempotence
    u2 = oracle.project(g, u1, v1, w1, dt_over_rho0=s)
    assert max(np.abs(a - b).max() for a, b in zip(u2[:3], (u1, v1, w1))) < 1e-12
    # Pythagoras in the face-volume inner product (wall faces are zero in the synthetic input)
    gp = tuple(s * x for x in oracle.gradient(g, p))
    lhs = face_inner(g, u, u)
    rhs = face_inner(g, (u1, v1, w1), (u1, v1, w1)) + face_inner(g, gp, gp)
    assert abs(lhs - rhs) < 1e-12 * lhs
    assert abs(face_inner(g, (u1, v1, w1), gp)) < 1e-12 * lhs
    # linearity
    ub = synth.random_velocity(n, bc, 6)
    pa = oracle.project(g, *u)[3]
    pb = oracle.project(g, *ub)[3]
    pab = oracle.project(g, *(2.0 * x - 3.0 * y for x, y in zip(u, ub)))[3]
    assert rel(pab, 2.0 * pa - 3.0 * pb) < 1e-12


def test_translation_and_swap_symmetry():
    n = (8, 8, 6)
    bc = ("P", "P", "NN")
    g = Grid(*n, 0.125, 0.125, np.full(6, 1.0 / 6), bc)
    r = np.random.default_rng(2)
    f = r.standard_normal(g.shape)
    p, _ = oracle.poisson_solve(g, f)
    ps, _ = oracle.poisson_solve(g, np.roll(np.roll(f, 3, axis=2), -2, axis=1))
    assert np.abs(ps - np.roll(np.roll(p, 3, axis=2), -2, axis=1)).max() < 1e-12 * np.abs(p).max()
    pt, _ = oracle.poisson_solve(g, np.swapaxes(f, 1, 2))
    assert np.abs(pt - np.swapaxes(p, 1, 2)).max() < 1e-12 * np.abs(p).max()


def test_singular_rhs_defect_reported():
    g = Grid(4, 4, 4, 0.25, 0.25, np.full(4, 0.25), ("P", "NN", "NN"))
    f = np.full(g.shape, 2.5)
    p, info = oracle.poisson_solve(g, f)
    assert abs(info["compat_defect"] - 2.5) < 1e-14
    assert np.abs(p).max() < 1e-13


# ---- extension (§3.6) -----------------------------------------------------------------------------------

def droplet_case(n, bc, seed=1):
    C, centre = synth.droplet(n, bc, seed)
    g = Grid(*n, 1.0 / n[0], 1.0 / n[1], synth.uniform_dz(n[2]), bc)
    return g, C, centre


@pytest.mark.parametrize("mode", [0, 1])
def test_extension_exact_decomposition_and_static_droplet(mode):
    n = (24, 24, 20)
    bc = ("P", "P", "NN")
    g, C, _ = droplet_case(n, bc)
    rho1, rho2 = 100.0, 1.0
    mdot = np.ones(g.shape)
    s = oracle.stefan_source(g, C, mdot, rho1, rho2, mode)
    psi, _ = oracle.poisson_solve(g, s)
    gpsi = oracle.gradient(g, psi)
    udf = oracle.project(g, *synth.random_velocity(n, bc, 9))[:3]
    u = tuple(a + b for a, b in zip(udf, gpsi))
    out = oracle.extend_liquid_velocity(g, *u, C, mdot, rho1, rho2, mode)
    for a in range(3):
        assert np.abs(out[a] - udf[a]).max() < 1e-12 * max(1.0, np.abs(udf[a]).max())
    assert np.abs(oracle.divergence(g, *out[:3])).max() < 1e-10
    # static droplet: u is the Stefan flow only -> u1e = 0, uG = -(mdot/rho1) n on faces (§4.1)
    st = oracle.extend_liquid_velocity(g, *gpsi, C, mdot, rho1, rho2, mode)
    _, nrm = oracle.delta_and_normal(g, C, mode)
    for a in range(3):
        assert np.abs(st[a]).max() < 1e-12
        expect = -(1.0 / rho1) * oracle.interface.face_average(g, nrm[a], a)
        assert np.abs(st[3 + a] - expect).max() < 1e-12


@pytest.mark.parametrize("mode", [0, 1])
def test_planar_interface_normal_and_delta(mode):
    # C depends on x only, linear in the interior: |grad C| = slope, n = -sign(slope) e_x
    n = (16, 4, 5)
    g = Grid(*n, 0.1, 0.1, np.full(5, 0.1), ("NN", "P", "NN"))
    x = (np.arange(16) + 0.5) * 0.1
    C = np.broadcast_to(0.2 + 0.03 * x, g.shape).copy()
    mag, nrm = oracle.delta_and_normal(g, C, mode)
    assert np.allclose(mag[:, :, 1:-1], 0.03, rtol=1e-13)
    assert np.allclose(nrm[0][:, :, 1:-1], -1.0) and np.abs(nrm[1]).max() == 0 and np.abs(nrm[2]).max() == 0
    # clipping where min(C, 1 - C) < 1e-8
    C2 = C.copy()
    C2[:, :, 5] = 1.0 - 1e-9
    _, n2 = oracle.delta_and_normal(g, C2, mode)
    assert np.all(n2[0][:, :, 5] == 0.0)


def test_surface_integral_of_delta_is_sphere_area():
    # sum |grad C| dV approximates the interface area (the perimeter formula of §4.1 in 3-D); the interface
    # width is 1.5 cells, so the error falls roughly as dx^2 under refinement
    errs = []
    for N in (48, 96):
        g, C, _ = droplet_case((N, N, N), ("P", "P", "NN"), seed=4)
        mag, _ = oracle.delta_and_normal(g, C, 0)
        area = (mag * g.cell_volumes()).sum()
        errs.append(abs(area / (4 * math.pi * 0.15 ** 2) - 1.0))
    assert errs[1] < 0.02 and errs[1] < errs[0] / 3.0


def test_stretched_grid_generator():
    dz = synth.stretched_dz(64)
    r = dz[1:] / dz[:-1]
    assert abs(dz.sum() - 1.0) < 1e-13
    assert abs(np.max(np.maximum(r, 1 / r)) - 1.05) < 1e-9
    assert dz[0] < dz[32]


def test_paper_constants_fixture():
    with open(os.path.join(GOLDEN, "paper_constants.json")) as fh:
        c = json.load(fh)
    assert c["normal_clip"]["value"] == 1e-8
    assert 100 in c["density_ratios"]["value"]


@pytest.mark.parametrize("bc", Z_BCS)
@pytest.mark.parametrize("n", [1, 2, 3, 8, 31, 250])
def test_oracle_basis_diagonalises_stencil(bc, n):
    # the oracle's x/y basis must be orthonormal and diagonalise the stencil matrix to roundoff
    from oracle.poisson import _eig_axis
    w = np.full(n, 0.01)
    lam, Q = _eig_axis(w, bc)
    A = oracle.operator_matrix_1d(w, bc)
    assert np.abs(Q.T @ Q - np.eye(n)).max() < 1e-13
    assert np.abs(Q.T @ A @ Q - np.diag(lam)).max() <= 1e-12 * max(np.abs(A).max(), 1.0)


# ---- ND / DN on the transformed axes (x, y) ---------------------------------------------------------------

QUARTER_XY = list(itertools.product(("ND", "DN", "NN"), ("DN", "ND", "DD"), Z_BCS))


@pytest.mark.parametrize("bcx,bcy,bcz", QUARTER_XY)
def test_quarter_wave_xy_closed_form_and_dense_lu(bcx, bcy, bcz):
    """ND / DN ends on x and y: the closed-form eigenfunctions cos / sin(pi (2m+1)(j+1/2) / (2n)) are
    recovered, and the oracle matches the dense LU solve of the 3-D stencil."""
    n = (8, 6, 10)
    h = (0.125, 0.2, 0.1)
    g = Grid(*n, h[0], h[1], np.full(n[2], h[2]), (bcx, bcy, bcz))
    r = np.random.default_rng(zlib.crc32(("q" + bcx + bcy + bcz).encode()))
    f = np.zeros(g.shape)
    pstar = np.zeros(g.shape)
    for _ in range(3):
        ms = [int(r.integers(0, n[a])) for a in range(3)]
        parts = [basis_1d(b, n[a], ms[a]) for a, b in enumerate((bcx, bcy, bcz))]
        mode = parts[2][0][:, None, None] * parts[1][0][None, :, None] * parts[0][0][None, None, :]
        lam = sum(parts[a][1] / h[a] ** 2 for a in range(3))
        c = r.standard_normal()
        pstar += c * mode
        f += c * lam * mode
    p, _ = oracle.poisson_solve(g, f)
    assert rel(p, pstar) < 1e-12
    rr = np.random.default_rng(9)
    for nn in BRUTE_SIZES:
        dz = rr.uniform(0.5, 1.5, nn[2]) / nn[2]
        gg = Grid(*nn, 1.0 / nn[0], 0.7 / nn[1], dz, (bcx, bcy, bcz))
        ff = rr.standard_normal(gg.shape)
        assert rel(oracle.poisson_solve(gg, ff)[0], brute_solve(gg, ff)) < 1e-11, nn


# ---- Youngs gradient and face values (§3.2 Youngs' method; §3.6 Eq. int_vel) ---------------------------------

def _quadratic(r):
    """Random quadratic a + b t + c t^2 with its value and its exact first and second derivatives."""
    a, b, c = r.uniform(-1.0, 1.0, 3)
    return (lambda t: a + b * t + c * t * t), (lambda t: b + 2 * c * t), 2 * c


def test_youngs_gradient_closed_form_on_quadratic_product():
    """For C = f(x) g(y) h(z) with quadratic factors sampled at cell centres of a uniform grid, Youngs'
    corner average gives exactly d/dx C = f'(x) (g + dy^2 g''/4)(h + dz^2 h''/4) in every cell whose
    3x3x3 neighbourhood is inside the grid: the two x face differences around the cell average to the
    centred difference, exact for a quadratic, and each transverse corner average is the (1, 2, 1) / 4
    filter, which adds d^2/4 times the second derivative.  A (1, 1) / 2 transverse average, a dropped
    transverse average or a one-sided face difference each miss it."""
    r = np.random.default_rng(20190701)
    n = (9, 8, 7)
    h = (0.11, 0.07, 0.13)
    g = Grid(*n, h[0], h[1], np.full(n[2], h[2]), ("NN", "DD", "NN"))
    xs = [(np.arange(n[a]) + 0.5) * h[a] for a in range(3)]
    fs = [_quadratic(r) for _ in range(3)]
    val = [fs[a][0](xs[a]) for a in range(3)]
    der = [fs[a][1](xs[a]) for a in range(3)]
    smooth = [val[a] + h[a] ** 2 / 4.0 * fs[a][2] for a in range(3)]
    C = val[2][:, None, None] * val[1][None, :, None] * val[0][None, None, :]
    gx, gy, gz = oracle.grad_c(g, C, mode=1)
    ex = smooth[2][:, None, None] * smooth[1][None, :, None] * der[0][None, None, :]
    ey = smooth[2][:, None, None] * der[1][None, :, None] * smooth[0][None, None, :]
    ez = der[2][:, None, None] * smooth[1][None, :, None] * smooth[0][None, None, :]
    inner = (slice(1, -1),) * 3
    for got, want in ((gx, ex), (gy, ey), (gz, ez)):
        assert np.abs(got[inner] - want[inner]).max() < 1e-13 * np.abs(want).max()
    # the central-difference default has no transverse smoothing: f'(x) g(y) h(z)
    cx = oracle.grad_c(g, C, mode=0)[0]
    want0 = val[2][:, None, None] * val[1][None, :, None] * der[0][None, None, :]
    assert np.abs(cx[inner] - want0[inner]).max() < 1e-13 * np.abs(want0).max()


def test_youngs_gradient_closed_form_periodic_wave():
    """On an all-periodic grid C = cos(a x) cos(b y) cos(c z) has, in every cell (wrap-around included),
    the Youngs x derivative -sin(a x) sin(a dx)/dx * cos(b y) cos^2(b dy/2) * cos(c z) cos^2(c dz/2):
    centred face differences and a (1, 2, 1) / 4 filter (= cos^2 of half the phase step) per transverse
    axis."""
    n = (8, 6, 10)
    L = (1.0, 0.9, 1.3)
    h = tuple(L[a] / n[a] for a in range(3))
    g = Grid(*n, h[0], h[1], np.full(n[2], h[2]), ("P", "P", "P"))
    k = (2 * math.pi * 3 / L[0], 2 * math.pi * 1 / L[1], 2 * math.pi * 2 / L[2])
    xs = [(np.arange(n[a]) + 0.5) * h[a] for a in range(3)]
    cs = [np.cos(k[a] * xs[a]) for a in range(3)]
    ds = [-np.sin(k[a] * xs[a]) * math.sin(k[a] * h[a]) / h[a] for a in range(3)]
    ss = [cs[a] * math.cos(k[a] * h[a] / 2) ** 2 for a in range(3)]
    C = cs[2][:, None, None] * cs[1][None, :, None] * cs[0][None, None, :]
    got = oracle.grad_c(g, C, mode=1)
    want = (ss[2][:, None, None] * ss[1][None, :, None] * ds[0][None, None, :],
            ss[2][:, None, None] * ds[1][None, :, None] * ss[0][None, None, :],
            ds[2][:, None, None] * ss[1][None, :, None] * ss[0][None, None, :])
    for a in range(3):
        assert np.abs(got[a] - want[a]).max() < 1e-12 * max(np.abs(want[a]).max(), 1.0)


def _youngs_by_corners(grid, C):
    """Youngs' method written corner by corner: at each of the 8 corners of a cell, the derivative along an
    axis is the mean of the 4 differences across that axis inside the 2x2x2 block of cells sharing the
    corner (each over its centre distance); the cell value is the mean over its 8 corners.  Ghost cells copy
    C at bounded ends and wrap at periodic ones."""
    nx, ny, nz = grid.n
    w = grid.widths

    def cell(a, i):
        n = grid.n[a]
        if 0 <= i < n:
            return i
        if grid.bc[a] == "P":
            return i % n
        return 0 if i < 0 else n - 1

    def centre_dist(a, i):
        # distance between the centres of cells i and i + 1 (either may be a ghost)
        n = grid.n[a]
        wa = w[a]
        if grid.bc[a] == "P":
            return 0.5 * (wa[i % n] + wa[(i + 1) % n])
        if i < 0:
            return wa[0]
        if i >= n - 1:
            return wa[n - 1]
        return 0.5 * (wa[i] + wa[i + 1])

    out = [np.zeros(grid.shape) for _ in range(3)]
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                acc = [0.0, 0.0, 0.0]
                for sx in (0, 1):
                    for sy in (0, 1):
                        for sz in (0, 1):
                            lo = (i - 1 + sx, j - 1 + sy, k - 1 + sz)   # low cell of the 2x2x2 block
                            for a in range(3):
                                d = 0.0
                                for t1 in (0, 1):
                                    for t2 in (0, 1):
                                        idx_lo = list(lo)
                                        others = [b for b in range(3) if b != a]
                                        idx_lo[others[0]] += t1
                                        idx_lo[others[1]] += t2
                                        idx_hi = list(idx_lo)
                                        idx_hi[a] += 1
                                        clo = C[cell(2, idx_lo[2]), cell(1, idx_lo[1]), cell(0, idx_lo[0])]
                                        chi = C[cell(2, idx_hi[2]), cell(1, idx_hi[1]), cell(0, idx_hi[0])]
                                        d += (chi - clo) / centre_dist(a, idx_lo[a])
                                acc[a] += d / 4.0
                for a in range(3):
                    out[a][k, j, i] = acc[a] / 8.0
    return out


@pytest.mark.parametrize("bc", [("P", "NN", "DD"), ("NN", "P", "P"), ("DD", "DD", "ND")])
def test_youngs_gradient_matches_corner_by_corner_definition(bc):
    """The oracle's separable Youngs filter equals the corner-by-corner definition on every cell, boundary
    cells and a stretched z axis included."""
    r = np.random.default_rng(3)
    n = (5, 4, 6)
    dz = r.uniform(0.6, 1.4, n[2]) / n[2]
    g = Grid(*n, 0.2, 0.25, dz, bc)
    C = r.uniform(0.0, 1.0, g.shape)
    got = oracle.grad_c(g, C, mode=1)
    want = _youngs_by_corners(g, C)
    for a in range(3):
        assert np.abs(got[a] - want[a]).max() < 1e-12 * np.abs(want[a]).max()


@pytest.mark.parametrize("bc", [("NN", "P", "DD"), ("P", "DD", "NN")])
def test_face_average_of_linear_field_is_value_at_face(bc):
    """Face values of a cell field (the mdot_f and n_f of Eq. int_vel): for q linear in space on a uniform
    grid, every interior face (index i = low face of cell i, at x = i dx) carries q at the face position;
    the periodic face 0 averages the last and first cells; a bounded axis' end faces copy their one
    cell.  A half-cell offset (the mean of cells i and i + 1, or the cell value itself) fails."""
    from oracle.interface import face_average
    n = (6, 5, 7)
    h = (0.1, 0.2, 0.15)
    g = Grid(*n, h[0], h[1], np.full(n[2], h[2]), bc)
    coef = (0.7, -1.3, 2.1)
    xs = [(np.arange(n[a]) + 0.5) * h[a] for a in range(3)]
    q = 0.4 + coef[0] * xs[0][None, None, :] + coef[1] * xs[1][None, :, None] + coef[2] * xs[2][:, None, None]
    np_ax = (2, 1, 0)
    for a in range(3):
        f = face_average(g, q, a)
        faces = np.arange(f.shape[np_ax[a]]) * h[a]
        shape = [1, 1, 1]
        shape[np_ax[a]] = -1
        # value at the face: replace the coordinate of axis a by the face position
        others = 0.4 + sum(coef[b] * xs[b].reshape([-1 if np_ax[b] == d else 1 for d in range(3)])
                           for b in range(3) if b != a)
        at_face = others + coef[a] * faces.reshape(shape)
        nf = f.shape[np_ax[a]]
        interior = [slice(None)] * 3
        interior[np_ax[a]] = slice(1, n[a])
        interior = tuple(interior)
        assert np.abs(f[interior] - np.broadcast_to(at_face, f.shape)[interior]).max() < 1e-13
        first = np.take(f, [0], axis=np_ax[a])
        if g.bc[a] == "P":
            assert nf == n[a]
            want = 0.5 * (np.take(q, [0], axis=np_ax[a]) + np.take(q, [n[a] - 1], axis=np_ax[a]))
            assert np.abs(first - want).max() < 1e-14
        else:
            assert nf == n[a] + 1
            assert np.array_equal(first, np.take(q, [0], axis=np_ax[a]))
            assert np.array_equal(np.take(f, [n[a]], axis=np_ax[a]), np.take(q, [n[a] - 1], axis=np_ax[a]))


@pytest.mark.parametrize("mode", [0, 1])
def test_interface_velocity_with_linear_mdot_on_planar_ramp(mode):
    """Eq. int_vel on a linear volume-fraction ramp C = c0 + g.x (both gradient stencils exact, so
    n = -g/|g| in every cell whose neighbours are inside the grid) with mdot linear in x: on every face
    between two such cells uG - u1e = -(mdot(face)/rho1) n, mdot taken at the face position itself (x faces
    at i dx, y and z faces at the cell's own x).  A face value offset by half a cell, a wrong normal sign or
    rho2 in place of rho1 fails."""
    n = (10, 9, 8)
    h = (0.1, 0.1, 0.1)
    g = Grid(*n, h[0], h[1], np.full(n[2], h[2]), ("NN", "NN", "NN"))
    xs = [(np.arange(n[a]) + 0.5) * h[a] for a in range(3)]
    grad = np.array([0.05, -0.08, 0.03])
    C = 0.5 + grad[0] * (xs[0][None, None, :] - 0.5) + grad[1] * (xs[1][None, :, None] - 0.45) \
        + grad[2] * (xs[2][:, None, None] - 0.4)
    assert C.min() > 0.3 and C.max() < 0.7
    mdot = 1.0 + 0.6 * xs[0][None, None, :] + 0.0 * C
    rho1, rho2 = 50.0, 2.0
    zero = [np.zeros(oracle.face_shape(g, a)) for a in range(3)]
    out = oracle.extend_liquid_velocity(g, *zero, C, mdot, rho1, rho2, mode)
    nvec = -grad / np.linalg.norm(grad)
    # x faces i = 2..n-2 lie between interior cells i-1, i (both in 1..n-2); mdot there = 1 + 0.6 i dx
    fx = np.arange(n[0] + 1) * h[0]
    dx_ = out[3] - out[0]
    want_x = -(1.0 + 0.6 * fx)[None, None, :] / rho1 * nvec[0]
    sl = (slice(1, -1), slice(1, -1), slice(2, n[0] - 1))
    assert np.abs(dx_[sl] - np.broadcast_to(want_x, dx_.shape)[sl]).max() < 1e-14
    # y and z faces: mdot at the cell's own x
    want_yz = -(1.0 + 0.6 * xs[0])[None, None, :] / rho1
    dy_ = out[4] - out[1]
    sl = (slice(1, -1), slice(2, n[1] - 1), slice(1, -1))
    assert np.abs(dy_[sl] - np.broadcast_to(want_yz * nvec[1], dy_.shape)[sl]).max() < 1e-14
    dz_ = out[5] - out[2]
    sl = (slice(2, n[2] - 1), slice(1, -1), slice(1, -1))
    assert np.abs(dz_[sl] - np.broadcast_to(want_yz * nvec[2], dz_.shape)[sl]).max() < 1e-14
