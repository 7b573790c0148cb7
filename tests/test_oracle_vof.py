"""Pins of the oracle's VoF update (§3.1: the directional split of Eq. fluxes with the correction and implicit
volume deflation of Eq. final_corr_2; upwind fluxes stand in for the MTHINC ones the paper cites), on the CPU:

* a uniform C stays uniform under any interface velocity, divergent or not (the discrete form of
  dC/dt + div(uG C) = C div(uG) at constant C) -- breaks if the deflation term, the implicit split or the sign
  of the correction is wrong;
* with a discretely divergence-free uG on a periodic grid the liquid volume sum(C V) is conserved to roundoff
  -- breaks if the correction F uses the wrong split stages or sign;
* at a Courant number of one a uniform velocity along an axis moves C by exactly one cell (the upwind flux
  and its direction), and a diagonal one by one cell along each axis (each split step takes the previous
  step's result);
* a 2-D droplet evaporating at a constant mass flux, advected by the interface velocity of the §3.6
  extension, follows the diameter law of Eq. diam_cmflux (§4.1), with an error that falls as the grid is
  refined -- breaks if the deflation term is dropped or has the wrong sign, or if uG takes the wrong normal.
"""
import numpy as np
import pytest

import oracle
from oracle.vof import vof_update
from paper_1907_00890_gb300 import synth


@pytest.mark.parametrize("bc", [("P", "P", "P"), ("P", "NN", "P"), ("NN", "DD", "NN"), ("DD", "P", "ND")])
def test_uniform_volume_fraction_stays_uniform(bc):
    n = (10, 8, 6)
    dz = synth.stretched_dz(n[2], 1.05) if bc[2] != "P" else synth.uniform_dz(n[2])
    g = oracle.Grid(*n, 1.0 / n[0], 1.0 / n[1], dz, bc)
    u, v, w = synth.random_velocity(n, bc, 5, sigma=0.3)
    out = vof_update(g, np.full(g.shape, 0.37), u, v, w, 0.01)
    assert np.abs(out - 0.37).max() < 1e-14


@pytest.mark.parametrize("seed", [1, 2])
def test_volume_conserved_for_divergence_free_interface_velocity(seed):
    n = (12, 10, 8)
    bc = ("P", "P", "P")
    g = oracle.Grid(*n, 1.0 / n[0], 1.0 / n[1], synth.uniform_dz(n[2]), bc)
    udf = oracle.project(g, *synth.random_velocity(n, bc, 7 + seed, sigma=0.5))[:3]
    C = synth.rng(seed).uniform(0, 1, g.shape)
    V = g.cell_volumes()
    out = vof_update(g, C, *udf, 0.01)
    assert abs(((out - C) * V).sum()) < 1e-14 * (C * V).sum()
    assert np.abs(out - C).max() > 1e-4  # the step does move C


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_courant_one_translation(axis):
    n = (10, 8, 6)
    g = oracle.Grid(*n, 0.1, 0.125, np.full(n[2], 1.0 / 6), ("P", "P", "P"))
    C = synth.rng(3).uniform(0, 1, g.shape)
    h = (0.1, 0.125, 1.0 / 6)[axis]
    dt = 0.05
    vel = [np.zeros(g.shape) for _ in range(3)]
    vel[axis][:] = h / dt
    out = vof_update(g, C, *vel, dt)
    assert np.abs(out - np.roll(C, 1, axis=2 - axis)).max() < 1e-14


def test_courant_one_diagonal_translation():
    n = (10, 8, 6)
    h = (0.1, 0.125, 1.0 / 6)
    g = oracle.Grid(*n, h[0], h[1], np.full(n[2], h[2]), ("P", "P", "P"))
    C = synth.rng(4).uniform(0, 1, g.shape)
    dt = 0.05
    vel = [np.full(g.shape, h[a] / dt) for a in range(3)]
    out = vof_update(g, C, *vel, dt)
    assert np.abs(out - np.roll(C, (1, 1, 1), axis=(0, 1, 2))).max() < 1e-14


def _evaporating_droplet_diameter(N, shrink=0.1, rho1=10.0, rho2=1.0, m0=1.0):
    """Diameter (from the liquid volume) of a circular droplet, d0 = L/4, in an x-z plane with zero-pressure
    (DD) boundaries, after evaporating at the constant mass flux m0 long enough for Eq. diam_cmflux to shrink
    it by the fraction ``shrink``; returns (d0 measured, d measured, d from Eq. diam_cmflux)."""
    L, d0 = 1.0, 0.25
    dx = L / N
    g = oracle.Grid(N, 1, N, dx, dx, np.full(N, dx), ("DD", "P", "DD"))
    xc = (np.arange(N) + 0.5) * dx
    r = np.sqrt((xc[:, None, None] - 0.5 * L) ** 2 + (xc[None, None, :] - 0.5 * L) ** 2)
    C = 0.5 * (1.0 - np.tanh((r - 0.5 * d0) / (1.5 * dx)))
    V = g.cell_volumes()
    mdot = np.full(g.shape, m0)
    dt = 2.0 * dx  # interface speed m0 / rho1 = 0.1: Courant number 0.2
    t_end = shrink * d0 * rho1 / (2.0 * m0)
    steps = int(round(t_end / dt))
    diameter = lambda q: np.sqrt(4.0 * (q * V).sum() / (dx * np.pi))
    d_start = diameter(C)
    for _ in range(steps):
        # the one-fluid velocity of a static droplet is the Stefan flow alone (its liquid velocity is zero)
        psi, _ = oracle.poisson_solve(g, oracle.stefan_source(g, C, mdot, rho1, rho2))
        ext = oracle.extend_liquid_velocity(g, *oracle.gradient(g, psi), C, mdot, rho1, rho2)
        C = vof_update(g, C, *ext[3:6], dt)
    return d_start, diameter(C), d_start * (1.0 - 2.0 * m0 / (d_start * rho1) * steps * dt)


def test_evaporating_droplet_follows_diameter_law():
    errs = []
    for N in (32, 64):
        d_start, d, d_law = _evaporating_droplet_diameter(N)
        assert d < d_start  # the droplet shrinks
        errs.append(abs(d - d_law) / (d_start - d_law))  # error relative to the predicted shrink
    assert errs[1] < 0.05 and errs[1] < 0.5 * errs[0]
