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


def test_vof_workspace_overlap_refused(vp):
    """A workspace that overlaps C or C_out, even partly, is refused on the host before any launch."""
    import torch
    n = (8, 6, 5)
    bc = ("P", "P", "NN")
    plan = vp.Plan(n, 1.0 / 8, 1.0 / 6, synth.uniform_dz(5), bc)
    cells = 8 * 6 * 5
    big = torch.zeros(4 * cells, dtype=torch.float64, device="cuda")
    uG = [dev(a) for a in synth.random_velocity(n, bc, 3, sigma=0.1)]
    C = big[:cells].view(5, 6, 8)
    out = torch.empty(cells, dtype=torch.float64, device="cuda").view(5, 6, 8)
    before = vp.vofp_launch_count()
    for off in (cells // 2, cells - 1, 1):  # work starts inside C or ends inside it
        work = big[off:off + 2 * cells]
        with pytest.raises(RuntimeError):
            vp.vofp_vof_update(plan.handle, C, *uG, 1e-3, out, work)
    work = torch.empty(2 * cells, dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError):  # C_out inside the workspace
        vp.vofp_vof_update(plan.handle, C, *uG, 1e-3, work[cells // 3:cells // 3 + cells], work)
    assert vp.vofp_launch_count() == before
    vp.vofp_vof_update(plan.handle, C, *uG, 1e-3, out, work)  # disjoint: accepted
    plan.close()
