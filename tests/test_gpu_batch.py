"""GPU tests of the batched projection (one launch per pass over all instances, replayed as a CUDA graph).

* parity: every instance of a heterogeneous batch against the oracle (rel-L2 <= 1e-10), for FP32 transforms
  with refinement and for FP32-pair transforms; a batch of plans of different precisions is refused;
* batch invariance: an instance's result alone (batch of one) and in the batch agree to 1e-12 relative (far
  inside the 1e-10 bar; they are not bitwise equal because the FP64 reductions add block partials with
  atomics, whose order varies from run to run);
* graph replay: a second call on fresh inputs through the same graph agrees with the first to 1e-12;
* the 64-instance ensemble with per-axis sizes from {32, 48, 64, 96, 128, 160}: divergence-free output for
  all instances (oracle stencil) and oracle parity on a seeded sample of them.
"""
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
    nb = np.linalg.norm(np.ravel(b))
    return float(np.linalg.norm(np.ravel(a - b)) / nb) if nb > 0 else float(np.linalg.norm(np.ravel(a)))


CASES = [((32, 48, 40), ("P", "P", "NN")), ((48, 32, 64), ("P", "P", "NN")), ((20, 36, 24), ("NN", "DD", "DN")),
         ((64, 64, 32), ("P", "P", "P")), ((33, 17, 12), ("DD", "P", "ND")), ((96, 40, 20), ("P", "NN", "DD"))]


def make_instances(vp, cases, seed0, prec=None):
    prec = vp.MIXED if prec is None else prec
    insts = []
    for idx, (n, bc) in enumerate(cases):
        dz = synth.stretched_dz(n[2]) if bc[2] != "P" else synth.uniform_dz(n[2])
        g = oracle.Grid(*n, 1.0 / n[0], 1.0 / n[1], dz, bc)
        u0 = synth.random_velocity(n, bc, seed0 + idx)
        plan = vp.Plan(n, g.widths[0][0], g.widths[1][0], dz, bc, prec=prec,
                       max_refine=0 if prec == vp.FF else 6)
        insts.append(dict(g=g, u0=u0, plan=plan))
    return insts


def run_batch(vp, insts, dts):
    import torch
    b = vp.vofp_batch_create([it["plan"].handle for it in insts])
    us = [[dev(a) for a in it["u0"]] for it in insts]
    ps = [torch.empty(it["g"].shape, dtype=torch.float64, device="cuda") for it in insts]
    vp.vofp_batch_project(b, [x[0] for x in us], [x[1] for x in us], [x[2] for x in us], None, dts, ps)
    torch.cuda.synchronize()
    return b, us, ps


@pytest.mark.parametrize("precision", ["mixed", "ff"])
def test_batch_parity_invariance_and_replay(vp, precision):
    import torch
    insts = make_instances(vp, CASES, 500, vp.MIXED if precision == "mixed" else vp.FF)
    dts = [0.5, 1.0, 2.0, 0.25, 1.0, 0.1]
    b, us, ps = run_batch(vp, insts, dts)
    for it, u, p, dt in zip(insts, us, ps, dts):
        ou = oracle.project(it["g"], *it["u0"], dt_over_rho0=dt)
        assert rel(p.cpu().numpy(), ou[3]) < TOL
        for a in range(3):
            assert rel(u[a].cpu().numpy(), ou[a]) < TOL
    # the same instance alone in a batch of one gives the same bits
    for idx in (0, 2, 3):
        it = insts[idx]
        b1 = vp.vofp_batch_create([it["plan"].handle])
        u1 = [dev(a) for a in it["u0"]]
        p1 = torch.empty_like(ps[idx])
        vp.vofp_batch_project(b1, [u1[0]], [u1[1]], [u1[2]], None, [dts[idx]], [p1])
        torch.cuda.synchronize()
        assert rel(p1.cpu().numpy(), ps[idx].cpu().numpy()) < 1e-12
        for a in range(3):
            assert rel(u1[a].cpu().numpy(), us[idx][a].cpu().numpy()) < 1e-12
        vp.vofp_batch_destroy(b1)
    # replay the captured graph on fresh inputs written into the same buffers
    first = [p.clone() for p in ps]
    for it, u in zip(insts, us):
        for a in range(3):
            u[a].copy_(dev(it["u0"][a]))
    vp.vofp_batch_project(b, [x[0] for x in us], [x[1] for x in us], [x[2] for x in us], None, dts, ps)
    torch.cuda.synchronize()
    for p, q in zip(ps, first):
        assert rel(p.cpu().numpy(), q.cpu().numpy()) < 1e-12
    vp.vofp_batch_destroy(b)
    for it in insts:
        it["plan"].close()


def test_batch_refuses_mixed_precisions(vp):
    a = vp.Plan((16, 16, 16), 1 / 16, 1 / 16, synth.uniform_dz(16), ("P", "P", "NN"), prec=vp.MIXED)
    b = vp.Plan((16, 16, 16), 1 / 16, 1 / 16, synth.uniform_dz(16), ("P", "P", "NN"), prec=vp.FF)
    with pytest.raises(vp.VofpError):
        vp.vofp_batch_create([a.handle, b.handle])
    a.close()
    b.close()


@pytest.mark.parametrize("precision", ["mixed", "ff"])
def test_batch_64_instance_ensemble(vp, precision):
    import torch
    sizes = synth.batch_sizes(64)
    bc = ("P", "P", "NN")
    insts = make_instances(vp, [(n, bc) for n in sizes], 900, vp.MIXED if precision == "mixed" else vp.FF)
    dts = [1.0] * len(insts)
    b, us, ps = run_batch(vp, insts, dts)
    for it, u in zip(insts, us):
        d = oracle.divergence(it["g"], *[x.cpu().numpy() for x in u])
        d0 = oracle.divergence(it["g"], *it["u0"])
        assert np.abs(d).max() < 1e-10 * np.abs(d0).max()
    pick = synth.rng(7).choice(len(insts), size=5, replace=False)
    for idx in pick:
        it = insts[idx]
        ou = oracle.project(it["g"], *it["u0"], dt_over_rho0=1.0)
        assert rel(ps[idx].cpu().numpy(), ou[3]) < TOL
    vp.vofp_batch_destroy(b)
    for it in insts:
        it["plan"].close()


def test_tuned_plans_keep_parity(vp, tmp_path, monkeypatch):
    """Autotuned launch shapes change speed only: results stay within the parity bar, cache file written."""
    monkeypatch.setenv("VOFP_TUNE_CACHE", str(tmp_path / "tune.txt"))
    for n, bc, prec, tol in [((48, 40, 36), ("P", "P", "NN"), vp.MIXED, 1e-10),
                             ((40, 24, 30), ("NN", "P", "DN"), vp.FP64, 1e-12)]:
        dz = synth.stretched_dz(n[2])
        g = oracle.Grid(*n, 1.0 / n[0], 1.0 / n[1], dz, bc)
        f = synth.rng(5).standard_normal(g.shape)
        ref, _ = oracle.poisson_solve(g, f)
        plan = vp.Plan(n, g.widths[0][0], g.widths[1][0], dz, bc, prec=prec, tune=1)
        p = plan.poisson_solve(dev(f))
        assert rel(p.cpu().numpy(), ref) < tol
        plan.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-10), ("ff", 1e-10)])
def test_reversed_radix_order_keeps_parity(vp, tmp_path, monkeypatch, prec, tol):
    """The tuner's radix-order knob (stages of x and y in reverse order), forced through its cache file: same
    results to the parity bar on mixed-radix lengths (48 = 4 4 3, 40 = 2 4 5 -> reversed)."""
    import torch
    pr = {"fp64": vp.FP64, "mixed": vp.MIXED, "ff": vp.FF}[prec]
    n, bc = (48, 40, 36), ("P", "NN", "NN")
    key = "%s|%d|%d|%d|%d|%d|%d|%d" % (torch.cuda.get_device_name(0).replace(" ", "_"), n[0], n[1], n[2],
                                       vp.BC[bc[0]], vp.BC[bc[1]], vp.BC[bc[2]], pr)
    cache = tmp_path / "tune.txt"
    xpb = 8
    cache.write_text("%s %d %d %d %d\n" % (key, xpb, 8, -1 if prec != "fp64" else 0, 3))
    monkeypatch.setenv("VOFP_TUNE_CACHE", str(cache))
    dz = synth.stretched_dz(n[2])
    g = oracle.Grid(*n, 1.0 / n[0], 1.0 / n[1], dz, bc)
    f = synth.rng(9).standard_normal(g.shape)
    ref, _ = oracle.poisson_solve(g, f)
    plan = vp.Plan(n, g.widths[0][0], g.widths[1][0], dz, bc, prec=pr, tune=1)
    p = plan.poisson_solve(dev(f))
    assert rel(p.cpu().numpy(), ref) < tol
    plan.close()
