"""GPU parity of the VoF update with the interface velocity (vofp_vof_update: §3.1, Eqs. fluxes and
final_corr_2 with upwind fluxes) against the CPU oracle, element by element, FP64 (1e-12), on a droplet C and
a divergent interface velocity, over periodic and bounded axes with stretched z, up to the 128^3 droplet grid
the bench times (every cell compared); C_out over C."""
import numpy as np
import pytest

import oracle
from oracle.vof import vof_update
from paper_1907_00890_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_00890_gb300 import build
    build.build()
    from paper_1907_00890_gb300 import vofp
    return vofp


def dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("n,bc", [((24, 20, 16), ("P", "P", "NN")), ((17, 23, 12), ("NN", "DD", "P")),
                                  ((20, 9, 14), ("DD", "P", "ND")), ((1, 12, 10), ("NN", "P", "DN")),
                                  ((96, 80, 64), ("P", "P", "P")), ((128, 128, 128), ("P", "P", "NN"))])
def test_vof_update_vs_oracle(vp, n, bc):
    dz = synth.stretched_dz(n[2]) if bc[2] != "P" else synth.uniform_dz(n[2])
    g = oracle.Grid(*n, 1.0 / n[0], 1.0 / n[1], dz, bc)
    C, _ = synth.droplet(n, bc, 91, dz=dz)
    uG = synth.random_velocity(n, bc, 92, sigma=0.5)
    dt = 0.1 / max(n)  # Courant number well below one
    ref = vof_update(g, C, *uG, dt)
    plan = vp.Plan(n, g.widths[0][0], g.widths[1][0], dz, bc)
    Cd = dev(C)
    out = plan.vof_update(Cd, *[dev(a) for a in uG], dt)
    got = out.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-12 * max(np.abs(ref).max(), 1.0)
    plan.vof_update(Cd, *[dev(a) for a in uG], dt, out=Cd)  # in place
    assert np.abs(Cd.cpu().numpy() - ref).max() <= 1e-12 * max(np.abs(ref).max(), 1.0)
    plan.close()
