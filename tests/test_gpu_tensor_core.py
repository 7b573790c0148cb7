"""GPU parity of the tensor-core x passes (tcgen05, 3xTF32 dense transform-matrix products) of FP32 refinement
plans, switched on by VOFP_X_TC=1 at plan creation, against the CPU oracle.

Bars: the refined solve and the projection within 1e-10 of the oracle (the mixed-precision bar) for every x
boundary condition, power-of-two and other lengths; the plan holds the transform tables (more device memory
than the same plan without them), so the tensor-core passes are the ones that ran.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1907_00890_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-10


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


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def tc_plan(vp, n, g, bc, **kw):
    os.environ["VOFP_X_TC"] = "1"
    try:
        return vp.Plan(n, g.widths[0][0], g.widths[1][0], g.widths[2], bc, prec=vp.MIXED, **kw)
    finally:
        del os.environ["VOFP_X_TC"]


@pytest.mark.parametrize("n,bc", [((64, 40, 36), ("P", "P", "NN")), ((128, 64, 24), ("NN", "P", "DD")),
                                  ((100, 20, 24), ("DD", "NN", "P")), ((48, 30, 50), ("ND", "P", "NN")),
                                  ((96, 24, 20), ("DN", "DD", "ND"))])
def test_tensor_core_x_passes_vs_oracle(vp, n, bc):
    dz = synth.stretched_dz(n[2]) if bc[2] != "P" else synth.uniform_dz(n[2])
    g = oracle.Grid(*n, 1.0 / n[0], 0.9 / n[1], dz, bc)
    f = synth.rng(sum(n)).standard_normal(g.shape)
    ref, _ = oracle.poisson_solve(g, f)
    plan = tc_plan(vp, n, g, bc)
    plain = vp.Plan(n, g.widths[0][0], g.widths[1][0], dz, bc, prec=vp.MIXED)
    assert vp.vofp_plan_workspace_bytes(plan.handle) > vp.vofp_plan_workspace_bytes(plain.handle)
    plain.close()
    p, info = plan.poisson_solve(dev(f), info=True)
    assert rel(p.cpu().numpy(), ref) < TOL, info
    assert info["rel_residual"] <= TOL
    # the projection (divergence right-hand side, residual and inverse passes on the tensor cores)
    u0 = synth.random_velocity(n, bc, 3)
    ou = oracle.project(g, *u0, dt_over_rho0=0.5)
    u = [dev(a) for a in u0]
    pp = plan.project(*u, dt_over_rho0=0.5)
    assert rel(pp.cpu().numpy(), ou[3]) < TOL
    for a in range(3):
        assert rel(u[a].cpu().numpy(), ou[a]) < TOL
    plan.close()

