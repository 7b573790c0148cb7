"""Pins of the oracle's variable-density pressure step (§3.2, Eq. lap_p with its pressure-splitting term and
the velocity update after it) against facts the equations fix, on the CPU:

* constant density (rho1 = rho2): the splitting term vanishes and the step is the constant-coefficient
  projection;
* p^n = p^{n-1} = 0: the step is the constant-coefficient projection with dt / min(rho1, rho2);
* fixed point: when the extrapolated pressure p_hat is the pressure that makes u* divergence-free for the
  variable-coefficient operator -- u* = u_df + dt (1/rho_f) G P with D u_df = 0 and p_hat = P -- the split
  step returns p = P and u = u_df exactly (the splitting is exact at a steady pressure).  p^n and p^{n-1} are
  chosen so that the second-order extrapolation with dt / dt_prev gives P (a wrong extrapolation, sign, face
  density or mixture rule breaks it).  The face density here is written independently of the oracle's.

And of the boiling variant (Appendix A, the interface velocity from the vapour-velocity extension):

* exchanging the phases (C -> 1 - C, mdot -> -mdot, rho1 <-> rho2) turns it into the liquid extension of
  §3.6, pinned in test_oracle_pins.py;
* a pure Stefan flow (a static bubble) extends to zero and gives uG = -(mdot_f / rho2) n_f.
"""
import numpy as np
import pytest

import oracle
from oracle import Grid
from paper_1907_00890_gb300 import synth


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


CASES = [((10, 8, 6), ("P", "P", "NN")), ((9, 7, 6), ("NN", "DD", "P")), ((8, 6, 7), ("DD", "NN", "ND")),
         ((6, 9, 5), ("P", "NN", "DN")), ((7, 6, 8), ("DD", "P", "DD"))]


def grid_for(n, bc, seed):
    dz = synth.stretched_dz(n[2], 1.05) if bc[2] != "P" else synth.uniform_dz(n[2])
    return Grid(n[0], n[1], n[2], 1.0 / n[0], 1.0 / n[1], dz, bc)


def face_density(g, rho):
    """rho on the faces by edge padding: mean of the two cells across a face; a bounded end face takes the
    cell next to it (padding by a copy of it makes the 'mean' that cell)."""
    out = []
    for axis, npax in ((0, 2), (1, 1), (2, 0)):
        mode = "wrap" if g.bc[axis] == "P" else "edge"
        pad = [(0, 0)] * 3
        pad[npax] = (1, 1)
        rp = np.pad(rho, pad, mode=mode)
        n = g.n[axis]
        a = np.take(rp, np.arange(0, n + 1), axis=npax)
        b = np.take(rp, np.arange(1, n + 2), axis=npax)
        f = 0.5 * (a + b)
        if g.bc[axis] == "P":
            f = np.take(f, np.arange(0, n), axis=npax)
        out.append(f)
    return out


def vol_mean_free(g, q):
    V = np.asarray(g.widths[2])[:, None, None] * g.widths[0][0] * g.widths[1][0] * np.ones(g.shape)
    return q - (q * V).sum() / V.sum()


@pytest.mark.parametrize("n,bc", CASES)
def test_constant_density_is_plain_projection(n, bc):
    g = grid_for(n, bc, 1)
    rng = synth.rng(101)
    u, v, w = synth.random_velocity(n, bc, 102)
    C = rng.uniform(0, 1, g.shape)
    pn, pm = rng.standard_normal(g.shape), rng.standard_normal(g.shape)
    src = rng.standard_normal(g.shape)
    a = oracle.project_variable_density(g, u, v, w, C, pn, pm, 0.3, 0.4, 2.5, 2.5, src=src)
    b = oracle.project(g, u, v, w, src=src, dt_over_rho0=0.3 / 2.5)
    for x, y in zip(a[:4], b[:4]):
        assert rel(x, y) < 1e-12


@pytest.mark.parametrize("n,bc", CASES)
def test_zero_pressure_history_uses_the_smaller_density(n, bc):
    g = grid_for(n, bc, 2)
    rng = synth.rng(201)
    u, v, w = synth.random_velocity(n, bc, 202)
    C = rng.uniform(0, 1, g.shape)
    z = np.zeros(g.shape)
    a = oracle.project_variable_density(g, u, v, w, C, z, z, 0.2, 0.2, 50.0, 1.5)
    b = oracle.project(g, u, v, w, dt_over_rho0=0.2 / 1.5)
    for x, y in zip(a[:4], b[:4]):
        assert rel(x, y) < 1e-12


@pytest.mark.parametrize("n,bc", CASES)
@pytest.mark.parametrize("rho1,rho2", [(100.0, 1.0), (1.0, 20.0)])
def test_steady_pressure_is_a_fixed_point(n, bc, rho1, rho2):
    g = grid_for(n, bc, 3)
    rng = synth.rng(301)
    singular = all(b in ("P", "NN") for b in bc)
    # a discretely divergence-free velocity and a pressure P in the solver's gauge
    u0, v0, w0 = synth.random_velocity(n, bc, 302)
    udf = oracle.project(g, u0, v0, w0)[:3]
    P = rng.standard_normal(g.shape)
    if singular:
        P = vol_mean_free(g, P)
    C, _ = synth.droplet(n, bc, 303)
    rho = rho1 * C + rho2 * (1.0 - C)
    rf = face_density(g, rho)
    GP = oracle.gradient(g, P)
    dt, dt_prev = 0.05, 0.04
    ustar = [udf[a] + dt * GP[a] / rf[a] for a in range(3)]
    # p^n, p^{n-1} whose extrapolation (1 + r) p^n - r p^{n-1} with r = dt / dt_prev is P
    r = dt / dt_prev
    Q = rng.standard_normal(g.shape)
    pn = P + 0.3 * Q
    pm = P + 0.3 * Q * (1.0 + r) / r
    uo, vo, wo, p, _ = oracle.project_variable_density(g, *ustar, C, pn, pm, dt, dt_prev, rho1, rho2)
    assert rel(p, P) < 1e-10
    for x, y in zip((uo, vo, wo), udf):
        assert np.abs(x - y).max() < 1e-10 * max(np.abs(y).max(), 1.0)


# ---- the boiling variant (Appendix A): vapour-velocity extension ----------------------------------------

@pytest.mark.parametrize("n,bc", CASES[:3])
@pytest.mark.parametrize("mode", [0, 1])
def test_vapour_extension_is_the_phase_exchanged_liquid_extension(n, bc, mode):
    """Exchanging the phases (C -> 1 - C, mdot -> -mdot, rho1 <-> rho2) turns the vapour extension into the
    liquid one of §3.6, whose pins live in test_oracle_pins.py."""
    g = grid_for(n, bc, 4)
    C, _ = synth.droplet(n, bc, 401)
    mdot = 1.0 + 0.3 * synth.rng(402).standard_normal(g.shape)
    u, v, w = synth.random_velocity(n, bc, 403)
    a = oracle.extend_vapour_velocity(g, u, v, w, C, mdot, 1000.0, 1.5, mode=mode)
    b = oracle.extend_liquid_velocity(g, u, v, w, 1.0 - C, -mdot, 1.5, 1000.0, mode=mode)
    for x, y in zip(a[:7], b[:7]):
        assert np.abs(x - y).max() <= 1e-12 * max(np.abs(y).max(), 1.0)


@pytest.mark.parametrize("n,bc", CASES[:3])
def test_vapour_extension_of_a_pure_stefan_flow(n, bc):
    """u = grad(phi) (the Stefan flow alone, a static bubble): u2e = 0 and uG = -(mdot_f / rho2) n_f."""
    g = grid_for(n, bc, 5)
    C, _ = synth.droplet(n, bc, 501)
    mdot = np.full(g.shape, 0.7)
    rho1, rho2 = 1000.0, 1.5
    s = oracle.stefan_source(g, C, mdot, rho1, rho2)
    phi, _ = oracle.poisson_solve(g, s)
    u = oracle.gradient(g, phi)
    out = oracle.extend_vapour_velocity(g, *u, C, mdot, rho1, rho2)
    scale = max(np.abs(x).max() for x in u)
    for a in range(3):
        assert np.abs(out[a]).max() < 1e-12 * scale
    _, nrm = oracle.delta_and_normal(g, C)
    from oracle.interface import face_average
    for a in range(3):
        want = -0.7 / rho2 * face_average(g, nrm[a], a)
        assert np.abs(out[3 + a] - want).max() < 1e-12 * max(scale, 1.0)
