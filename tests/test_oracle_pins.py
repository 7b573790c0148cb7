"""Pins of the CPU oracle against facts fixed by the paper and by the mathematics (no GPU).

* closed-form discrete eigenfunctions of the MAC Laplacian per boundary condition (cos / sin bases);
* brute force: the full 3-D matrix of the stencil, solved by dense LU (bordered for the singular case);
* Green's identity, D G = L consistency, the 1-D matrices vs the 3-D stencil;
* projection invariants: zero-mean gauge, machine-epsilon divergence, idempotence, discrete Pythagoras,
  linearity, translation equivariance, x <-> y symmetry;
* the extension of §3.6: exact decomposition u = u_df + grad(psi), the static-droplet case of §4.1
  (u1e = 0, uG = -(mdot/rho1) n), divergence-free u1e (Eq. jump_subtr), planar-interface normals.
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
