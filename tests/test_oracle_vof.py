"""Pins of the oracle's VoF update (§3.1: the directional split of Eq. fluxes with the correction and implicit
volume deflation of Eq. final_corr_2; upwind fluxes stand in for the MTHINC ones the paper cites), on the CPU:

* a uniform C stays uniform under any interface velocity, divergent or not (the discrete form of
  dC/dt + div(uG C) = C div(uG) at constant C) -- breaks if the deflation term, the implicit split or the sign
  of the correction is wrong;
* with a discretely divergence-free uG on a periodic grid the liquid volume sum(C V) is conserved to roundoff
  -- breaks if the correction F uses the wrong split stages or sign;
* at a Courant number of one a uniform velocity along an axis moves C by exactly one cell (the upwind flux
  and its direction).
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
