"""GPU parity of the variable-density pressure step (vofp_project_vd: §3.2, Eq. lap_p with its pressure-splitting
term and the velocity update after it) against the CPU oracle, on seeded droplet inputs with the paper's
density ratio of 100 in both orders.

Bar: relative L2 <= 1e-12 for p and the three face arrays on FP64 plans; 1e-10 on the reduced-precision plans
(FP32 + FP64 refinement, FP32 pairs) -- the same bars as the constant-density projection.
"""
import numpy as np
import pytest

import oracle
from paper_1907_00890_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-12


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


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    nb = np.linalg.norm(np.ravel(b))
    return float(np.linalg.norm(np.ravel(a - b)) / nb) if nb > 0 else float(np.linalg.norm(np.ravel(a)))


def inputs(n, bc, seed, rho1, rho2, with_prev=True):
    dz = synth.stretched_dz(n[2]) if bc[2] != "P" else synth.uniform_dz(n[2])
    g = oracle.Grid(*n, 1.0 / n[0], 0.8 / n[1], dz, bc)
    C, _ = synth.droplet(n, bc, seed, dz=dz)
    u = synth.random_velocity(n, bc, seed + 1)
    r = synth.rng(seed + 2)
    pn = r.standard_normal(g.shape)
    pm = pn + 0.1 * r.standard_normal(g.shape) if with_prev else None
    src = oracle.stefan_source(g, C, np.ones(g.shape), rho1, rho2)
    return g, dz, C, u, pn, pm, src


CASES = [((26, 18, 22), ("P", "P", "NN")), ((37, 11, 13), ("NN", "DD", "P")), ((20, 24, 17), ("DD", "NN", "ND")),
         ((33, 16, 12), ("P", "DD", "DN")), ((24, 20, 18), ("NN", "NN", "NN")), ((31, 29, 16), ("P", "P", "DD"))]


@pytest.mark.parametrize("n,bc", CASES)
@pytest.mark.parametrize("rho1,rho2", [(100.0, 1.0), (1.0, 100.0)])
def test_project_vd_vs_oracle(vp, n, bc, rho1, rho2):
    g, dz, C, u0, pn, pm, src = inputs(n, bc, 31, rho1, rho2)
    dt, dt_prev = 2e-3, 2.5e-3
    ref = oracle.project_variable_density(g, *u0, C, pn, pm, dt, dt_prev, rho1, rho2, src=src)
    plan = vp.Plan(n, g.widths[0][0], g.widths[1][0], dz, bc)
    u = [dev(a) for a in u0]
    p, info = plan.project_vd(*u, dev(C), dev(pn), dev(pm), dt, dt_prev, rho1, rho2, src=dev(src), info=True)
    assert info["status"] in (0, 1)
    assert rel(host(p), ref[3]) < TOL
    for a in range(3):
        assert rel(host(u[a]), ref[a]) < TOL
    plan.close()


@pytest.mark.parametrize("n,bc", CASES[:3])
def test_project_vd_first_step_and_aliased_p(vp, n, bc):
    """No p^{n-1} (p_hat = p^n), and p^{n+1} written over the p^n buffer."""
    g, dz, C, u0, pn, _, src = inputs(n, bc, 41, 100.0, 1.0, with_prev=False)
    ref = oracle.project_variable_density(g, *u0, C, pn, None, 1e-3, 1.0, 100.0, 1.0, src=src)
    plan = vp.Plan(n, g.widths[0][0], g.widths[1][0], dz, bc)
    u = [dev(a) for a in u0]
    pbuf = dev(pn)
    plan.project_vd(*u, dev(C), pbuf, None, 1e-3, 1.0, 100.0, 1.0, src=dev(src), p=pbuf)
    assert rel(host(pbuf), ref[3]) < TOL
    for a in range(3):
        assert rel(host(u[a]), ref[a]) < TOL
    plan.close()


@pytest.mark.parametrize("precision", ["mixed", "ff"])
@pytest.mark.parametrize("n,bc", [((48, 40, 36), ("P", "P", "NN")), ((30, 26, 20), ("DD", "NN", "DN"))])
def test_project_vd_reduced_precisions(vp, precision, n, bc):
    g, dz, C, u0, pn, pm, src = inputs(n, bc, 51, 100.0, 1.0)
    ref = oracle.project_variable_density(g, *u0, C, pn, pm, 2e-3, 2e-3, 100.0, 1.0, src=src)
    prec = vp.MIXED if precision == "mixed" else vp.FF
    plan = vp.Plan(n, g.widths[0][0], g.widths[1][0], dz, bc, prec=prec, max_refine=6 if prec == vp.MIXED else 0)
    u = [dev(a) for a in u0]
    p = plan.project_vd(*u, dev(C), dev(pn), dev(pm), 2e-3, 2e-3, 100.0, 1.0, src=dev(src))
    assert rel(host(p), ref[3]) < 1e-10
    for a in range(3):
        assert rel(host(u[a]), ref[a]) < 1e-10
    plan.close()


def test_project_vd_rejects_bad_arguments(vp):
    n, bc = (8, 6, 5), ("P", "P", "NN")
    g, dz, C, u0, pn, pm, src = inputs(n, bc, 61, 100.0, 1.0)
    plan = vp.Plan(n, g.widths[0][0], g.widths[1][0], dz, bc)
    u = [dev(a) for a in u0]
    for args in ((0.0, 1.0, 100.0, 1.0), (1e-3, 0.0, 100.0, 1.0), (1e-3, 1e-3, -1.0, 1.0),
                 (1e-3, 1e-3, 100.0, float("inf"))):
        with pytest.raises(Exception):
            plan.project_vd(*u, dev(C), dev(pn), dev(pm), *args)
    # nothing was modified by the rejected calls
    for a in range(3):
        assert np.array_equal(host(u[a]), u0[a])
    plan.close()


# ---- the boiling variant (Appendix A): vapour-velocity extension ----------------------------------------

@pytest.mark.parametrize("n,bc", [((30, 26, 20), ("P", "P", "NN")), ((24, 28, 18), ("NN", "DD", "DN"))])
@pytest.mark.parametrize("precision", ["fp64", "ff"])
def test_extend_vapour_vs_oracle(vp, n, bc, precision):
    dz = synth.stretched_dz(n[2]) if bc[2] != "P" else synth.uniform_dz(n[2])
    g = oracle.Grid(*n, 1.0 / n[0], 0.8 / n[1], dz, bc)
    C, _ = synth.droplet(n, bc, 71, dz=dz)
    mdot = 1.0 + 0.2 * synth.rng(72).standard_normal(g.shape)
    u0 = synth.random_velocity(n, bc, 73)
    rho1, rho2 = 1000.0, 1.5
    ref = oracle.extend_vapour_velocity(g, *u0, C, mdot, rho1, rho2)
    prec = vp.FP64 if precision == "fp64" else vp.FF
    plan = vp.Plan(n, g.widths[0][0], g.widths[1][0], dz, bc, prec=prec, max_refine=0)
    out = plan.extend(*[dev(a) for a in u0], dev(C), dev(mdot), rho1, rho2, vapour=True)
    tol = TOL if prec == vp.FP64 else 1e-10
    for a in range(7):
        assert rel(host(out[a]), ref[a]) < tol, a
    plan.close()
