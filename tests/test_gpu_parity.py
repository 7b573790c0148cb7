"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the same seeded inputs.

Bar (FP64 path): relative L2 error <= 1e-12 for p / phi and every face array, both sides in the zero-mean
gauge.  Sizes span several transform tiles with ragged tails, odd and prime lengths, 1- and 2-cell axes,
every boundary-condition combination, stretched z, and the full 128^3 two-solve droplet workload.
"""
import itertools

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
    na = np.linalg.norm(np.ravel(a - b))
    return float(na / nb) if nb > 0 else float(na)


def make(n, bc, seed=0, stretched=False):
    dz = synth.stretched_dz(n[2]) if stretched else synth.uniform_dz(n[2])
    g = oracle.Grid(*n, 1.0 / n[0], 0.8 / n[1], dz, bc)
    return g, dz


XY = ("P", "NN", "DD")
ZB = ("P", "NN", "DD", "ND", "DN")


@pytest.mark.parametrize("bcx,bcy,bcz", list(itertools.product(XY, XY, ZB)))
def test_poisson_every_bc(vp, bcx, bcy, bcz):
    n = (20, 12, 9)
    bc = (bcx, bcy, bcz)
    g, dz = make(n, bc, stretched=bcz != "P")
    f = synth.rng(11).standard_normal(g.shape)
    ref, rinfo = oracle.poisson_solve(g, f)
    plan = vp.Plan(n, g.widths[0][0], g.widths[1][0], dz, bc)
    p, info = plan.poisson_solve(dev(f), info=True)
    assert rel(host(p), ref) < TOL
    assert abs(info["compat_defect"] - rinfo["compat_defect"]) < 1e-13
    plan.close()


SIZES = [(1, 1, 1), (1, 6, 8), (7, 1, 5), (2, 2, 2), (3, 5, 7), (37, 11, 13), (48, 20, 30), (20, 96, 3),
         (160, 12, 10), (64, 64, 64), (30, 28, 1), (250, 3, 4)]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("bc", [("P", "P", "NN"), ("NN", "DD", "P"), ("DD", "P", "DN")])
def test_poisson_sizes(vp, n, bc):
    g, dz = make(n, bc, stretched=bc[2] != "P")
    f = synth.rng(sum(n)).standard_normal(g.shape)
    ref, _ = oracle.poisson_solve(g, f)
    plan = vp.Plan(n, g.widths[0][0], g.widths[1][0], dz, bc)
    p = plan.poisson_solve(dev(f))
    assert rel(host(p), ref) < TOL, (n, bc)
    plan.close()


# lengths with a prime factor above 13 run the Bluestein (chirp-z) form: primes, 4 * 31, 2 * 3 * 41, 251,
# and 2039 (prime, Bluestein length 4096, the longest that takes it) on each transformed axis.  Convolution
# lengths (the least c * 2^k >= 2n - 1, c in {1, 3, 5, 15}): 17 -> 40, 37 -> 80, 97 -> 240, 124 -> 256,
# 246 and 251 -> 512, 2039 -> 4096
BLUESTEIN = [(17, 4, 3), (37, 13, 5), (124, 6, 4), (246, 17, 3), (251, 5, 2), (6, 97, 3), (4, 251, 3),
             (2039, 2, 2), (3, 2039, 2)]

# odd prime factors 7, 11 and 13 run their own stages (no Bluestein form): primes, prime powers, products of
# two of them and with powers of two and 3, on each transformed axis
ODD_PRIMES = [(7, 11, 3), (13, 5, 4), (49, 3, 2), (77, 26, 3), (143, 6, 2), (4, 121, 2), (5, 169, 2),
              (88, 104, 3), (231, 7, 2), (3, 1001, 2)]


@pytest.mark.parametrize("n", BLUESTEIN)
@pytest.mark.parametrize("bc", [("P", "P", "NN"), ("NN", "DD", "P"), ("DD", "NN", "DN")])
@pytest.mark.parametrize("precision", ["fp64", "ff"])
def test_poisson_bluestein_lengths(vp, n, bc, precision):
    g, dz = make(n, bc, stretched=bc[2] != "P")
    f = synth.rng(sum(n) + 7).standard_normal(g.shape)
    ref, _ = oracle.poisson_solve(g, f)
    prec = vp.FP64 if precision == "fp64" else vp.FF
    plan = vp.Plan(n, g.widths[0][0], g.widths[1][0], dz, bc, prec=prec, max_refine=0 if prec == vp.FF else 6)
    p = plan.poisson_solve(dev(f))
    assert rel(host(p), ref) < (TOL if prec == vp.FP64 else 1e-10), (n, bc)
    plan.close()


@pytest.mark.parametrize("n", ODD_PRIMES)
@pytest.mark.parametrize("bc", [("P", "P", "NN"), ("NN", "DD", "P"), ("DD", "NN", "DN")])
@pytest.mark.parametrize("precision", ["fp64", "mixed", "ff"])
def test_poisson_odd_prime_lengths(vp, n, bc, precision):
    g, dz = make(n, bc, stretched=bc[2] != "P")
    f = synth.rng(sum(n) + 11).standard_normal(g.shape)
    ref, _ = oracle.poisson_solve(g, f)
    prec = {"fp64": vp.FP64, "mixed": vp.MIXED, "ff": vp.FF}[precision]
    plan = vp.Plan(n, g.widths[0][0], g.widths[1][0], dz, bc, prec=prec, max_refine=0 if prec == vp.FF else 6)
    p = plan.poisson_solve(dev(f))
    assert rel(host(p), ref) < (TOL if prec == vp.FP64 else 1e-10), (n, bc)
    plan.close()


def test_poisson_in_place_and_side_stream(vp):
    import torch
    n = (33, 17, 12)
    bc = ("P", "NN", "NN")
    g, dz = make(n, bc)
    f = synth.rng(3).standard_normal(g.shape)
    ref, _ = oracle.poisson_solve(g, f)
    plan = vp.Plan(n, g.widths[0][0], g.widths[1][0], dz, bc)
    s = torch.cuda.Stream()
    t = dev(f)
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        plan.poisson_solve(t, p=t)
    s.synchronize()
    assert rel(host(t), ref) < TOL
    plan.close()


def test_project_small_config(vp):
    c = synth.config_small()
    g = oracle.Grid(*c["n"], c["dx"], c["dy"], c["dz"], c["bc"])
    ou, ov, ow, op, oi = oracle.project(g, c["u"], c["v"], c["w"], dt_over_rho0=c["dt_over_rho0"])
    plan = vp.Plan(c["n"], c["dx"], c["dy"], c["dz"], c["bc"])
    u, v, w = dev(c["u"]), dev(c["v"]), dev(c["w"])
    p, info = plan.project(u, v, w, dt_over_rho0=c["dt_over_rho0"], info=True)
    for a, b in ((p, op), (u, ou), (v, ov), (w, ow)):
        assert rel(host(a), b) < TOL
    d = oracle.divergence(g, host(u), host(v), host(w))
    assert np.abs(d).max() < 1e-12 * np.abs(oracle.divergence(g, c["u"], c["v"], c["w"])).max()
    assert info["status"] in (0, 1)
    plan.close()


@pytest.mark.parametrize("bc", [("P", "P", "NN"), ("DD", "NN", "ND"), ("NN", "P", "P")])
def test_project_source_scale_and_no_p(vp, bc):
    n = (26, 18, 22)
    g, dz = make(n, bc, stretched=bc[2] != "P")
    u0 = synth.random_velocity(n, bc, 21)
    src = synth.rng(22).standard_normal(g.shape)
    s = 0.0125
    ou = oracle.project(g, *u0, src=src, dt_over_rho0=s)
    plan = vp.Plan(n, g.widths[0][0], g.widths[1][0], dz, bc)
    u = [dev(a) for a in u0]
    p = plan.project(*u, src=dev(src), dt_over_rho0=s)
    assert rel(host(p), ou[3]) < TOL
    for a in range(3):
        assert rel(host(u[a]), ou[a]) < TOL
    u2 = [dev(a) for a in u0]
    plan.project(*u2, src=dev(src), dt_over_rho0=s, want_p=False)
    for a in range(3):
        assert rel(host(u2[a]), ou[a]) < TOL
    plan.close()


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("bc", [("P", "P", "NN"), ("NN", "DD", "DN"), ("P", "P", "P")])
def test_extend_droplet(vp, mode, bc):
    n = (40, 36, 30)
    g, dz = make(n, bc, stretched=bc[2] != "P")
    C, centre = synth.droplet(n, bc, 5, dz=dz)
    mdot = 1.0 + 0.1 * synth.rng(6).standard_normal(g.shape)
    u0 = synth.swirl_velocity(n, bc, centre, 7)
    ref = oracle.extend_liquid_velocity(g, *u0, C, mdot, 100.0, 1.0, mode=mode)
    plan = vp.Plan(n, g.widths[0][0], g.widths[1][0], dz, bc, grad_mode=mode)
    out = plan.extend(*[dev(a) for a in u0], dev(C), dev(mdot), 100.0, 1.0)
    for a in range(7):
        assert rel(host(out[a]), ref[a]) < TOL, a
    plan.close()


def test_droplet_step_128(vp):
    """The full two-solve step at 128^3: projection with the Stefan source, then the extension."""
    c = synth.config_droplet(128)
    g = oracle.Grid(*c["n"], c["dx"], c["dy"], c["dz"], c["bc"])
    s = oracle.stefan_source(g, c["C"], c["mdot"], c["rho1"], c["rho2"])
    ou = oracle.project(g, c["u"], c["v"], c["w"], src=s, dt_over_rho0=c["dt_over_rho0"])
    oe = oracle.extend_liquid_velocity(g, *ou[:3], c["C"], c["mdot"], c["rho1"], c["rho2"])
    plan = vp.Plan(c["n"], c["dx"], c["dy"], c["dz"], c["bc"])
    u, v, w = dev(c["u"]), dev(c["v"]), dev(c["w"])
    tC, tm = dev(c["C"]), dev(c["mdot"])
    assert rel(host(plan.stefan_source(tC, tm, c["rho1"], c["rho2"])), s) < TOL
    p = plan.project_stefan(u, v, w, tC, tm, c["rho1"], c["rho2"], dt_over_rho0=c["dt_over_rho0"])
    assert rel(host(p), ou[3]) < TOL
    for a, b in zip((u, v, w), ou[:3]):
        assert rel(host(a), b) < TOL
    out = plan.extend(u, v, w, tC, tm, c["rho1"], c["rho2"])
    for a in range(7):
        assert rel(host(out[a]), oe[a]) < TOL, a
    plan.close()


def test_info_defect_warning_and_nonfinite(vp):
    n = (16, 8, 8)
    bc = ("P", "NN", "NN")
    g, dz = make(n, bc)
    f = np.full(g.shape, 3.0)
    plan = vp.Plan(n, g.widths[0][0], g.widths[1][0], dz, bc)
    p, info = plan.poisson_solve(dev(f), info=True)
    assert info["status"] == 1 and abs(info["compat_defect"] - 3.0) < 1e-13
    assert np.abs(host(p)).max() < 1e-12
    f2 = synth.rng(1).standard_normal(g.shape)
    f2[3, 2, 1] = np.nan
    with pytest.raises(vp.VofpError) as e:
        plan.poisson_solve(dev(f2), info=True)
    assert e.value.status == -7
    plan.close()


def test_invalid_arguments_rejected_before_launch(vp):
    with pytest.raises(vp.VofpError):
        vp.Plan((0, 4, 4), 1.0, 1.0, np.ones(4), ("P", "P", "NN"))
    with pytest.raises(vp.VofpError):
        vp.Plan((4, 4, 4), 1.0, 1.0, np.array([1.0, -1.0, 1.0, 1.0]), ("P", "P", "NN"))
    with pytest.raises(vp.VofpError) as e:
        vp.Plan((5000, 4, 4), 1.0, 1.0, np.ones(4), ("P", "P", "NN"))  # axes up to 4096 cells
    assert e.value.status == -2
    plan = vp.Plan((4, 4, 4), 1.0, 1.0, np.ones(4), ("P", "P", "NN"))
    assert vp._lib.vofp_poisson_solve(plan.handle, None, None, None, None) == -1
    assert vp._lib.vofp_project(plan.handle, None, None, None, None, 1.0, None, None, None) == -1
    plan.close()


@pytest.mark.parametrize("n,bc,mode", [((128, 128, 128), ("P", "P", "NN"), 0), ((36, 30, 28), ("NN", "DD", "DN"), 1),
                                       ((33, 20, 24), ("P", "P", "P"), 0)])
def test_project_extend_step(vp, n, bc, mode):
    """vofp_project_extend (both solves of one step, shared geometry) against the oracle's two solves."""
    import torch
    dz = synth.stretched_dz(n[2]) if bc[2] != "P" else synth.uniform_dz(n[2])
    g = oracle.Grid(*n, 1.0 / n[0], 1.0 / n[1], dz, bc)
    C, centre = synth.droplet(n, bc, 12, dz=dz)
    mdot = 1.0 + 0.2 * synth.rng(13).standard_normal(g.shape)
    u0 = synth.swirl_velocity(n, bc, centre, 14)
    s = oracle.stefan_source(g, C, mdot, 100.0, 1.0, mode)
    dt = 0.01
    ou = oracle.project(g, *u0, src=s, dt_over_rho0=dt)
    oe = oracle.extend_liquid_velocity(g, *ou[:3], C, mdot, 100.0, 1.0, mode=mode)
    plan = vp.Plan(n, g.widths[0][0], g.widths[1][0], dz, bc, grad_mode=mode)
    u = [dev(a) for a in u0]
    p = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    ue = [torch.empty_like(a) for a in u]
    ug = [torch.empty_like(a) for a in u]
    phi = torch.empty_like(p)
    st, info = vp.vofp_project_extend(plan.handle, *u, dev(C), dev(mdot), 100.0, 1.0, dt, p, *ue, *ug, phi, info=True)
    assert rel(host(p), ou[3]) < TOL
    for a in range(3):
        assert rel(host(u[a]), ou[a]) < TOL
        assert rel(host(ue[a]), oe[a]) < TOL
        assert rel(host(ug[a]), oe[3 + a]) < TOL
    assert rel(host(phi), oe[6]) < TOL
    assert abs(info["compat_defect"] - ou[4]["compat_defect"]) < 1e-10 * max(1.0, abs(ou[4]["compat_defect"]))
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "ff"])
@pytest.mark.parametrize("pinned", [True, False])
def test_project_extend_host_buffers(vp, precision, pinned):
    """vofp_project_extend_host (host buffers in and out, transfers overlapped with the compute) against the
    oracle's two solves, twice in a row with the same plan (its device fields are reused), on pinned and on
    pageable host memory."""
    import torch
    n, bc = (36, 30, 28), ("P", "P", "NN")
    dz = synth.stretched_dz(n[2])
    g = oracle.Grid(*n, 1.0 / n[0], 1.0 / n[1], dz, bc)
    C, centre = synth.droplet(n, bc, 21, dz=dz)
    mdot = 1.0 + 0.2 * synth.rng(22).standard_normal(g.shape)
    u0 = synth.swirl_velocity(n, bc, centre, 23)
    s = oracle.stefan_source(g, C, mdot, 100.0, 1.0)
    ou = oracle.project(g, *u0, src=s, dt_over_rho0=0.01)
    oe = oracle.extend_liquid_velocity(g, *ou[:3], C, mdot, 100.0, 1.0)
    prec = vp.FP64 if precision == "fp64" else vp.FF
    tol = TOL if prec == vp.FP64 else 1e-10
    plan = vp.Plan(n, g.widths[0][0], g.widths[1][0], dz, bc, prec=prec, max_refine=0)

    def hostt(a):
        t = torch.tensor(np.ascontiguousarray(a), dtype=torch.float64)
        return t.pin_memory() if pinned else t

    ins = [hostt(a) for a in list(u0) + [C, mdot]]
    outs = [hostt(np.zeros_like(a)) for a in list(u0) + [C] + list(u0)]
    for _ in range(2):
        for t in outs:
            t.zero_()
        vp.vofp_project_extend_host(plan.handle, *ins, 100.0, 1.0, 0.01, *outs)
        torch.cuda.synchronize()
        for a in range(3):
            assert rel(outs[a].numpy(), ou[a]) < tol
            assert rel(outs[4 + a].numpy(), oe[3 + a]) < tol
        assert rel(outs[3].numpy(), ou[3]) < tol
    plan.close()


# ---- ND / DN on the transformed axes (quarter-wave transforms, DCT-IV / DST-IV) ---------------------------

QXY = list(itertools.product(("ND", "DN", "NN"), ("DN", "ND", "DD"), ZB))


@pytest.mark.parametrize("bcx,bcy,bcz", QXY)
def test_poisson_quarter_wave_xy(vp, bcx, bcy, bcz):
    n = (20, 12, 9)
    bc = (bcx, bcy, bcz)
    g, dz = make(n, bc, stretched=bcz != "P")
    f = synth.rng(13).standard_normal(g.shape)
    ref, _ = oracle.poisson_solve(g, f)
    plan = vp.Plan(n, g.widths[0][0], g.widths[1][0], dz, bc)
    assert rel(host(plan.poisson_solve(dev(f))), ref) < TOL
    plan.close()


@pytest.mark.parametrize("n", [(1, 6, 8), (7, 1, 5), (37, 17, 6), (31, 40, 5), (128, 96, 16), (250, 3, 4)])
@pytest.mark.parametrize("bc", [("ND", "DN", "NN"), ("DN", "P", "DD"), ("P", "ND", "P")])
@pytest.mark.parametrize("precision", ["fp64", "mixed", "ff"])
def test_poisson_quarter_wave_sizes(vp, n, bc, precision):
    g, dz = make(n, bc, stretched=bc[2] != "P")
    f = synth.rng(sum(n) + 17).standard_normal(g.shape)
    ref, _ = oracle.poisson_solve(g, f)
    prec = {"fp64": vp.FP64, "mixed": vp.MIXED, "ff": vp.FF}[precision]
    plan = vp.Plan(n, g.widths[0][0], g.widths[1][0], dz, bc, prec=prec, max_refine=0 if prec == vp.FF else 6)
    p = plan.poisson_solve(dev(f))
    assert rel(host(p), ref) < (TOL if prec == vp.FP64 else 1e-10), (n, bc)
    plan.close()


@pytest.mark.parametrize("bc", [("ND", "DN", "NN"), ("DN", "ND", "P")])
def test_project_and_extend_quarter_wave_xy(vp, bc):
    n = (26, 22, 14)
    g, dz = make(n, bc, stretched=bc[2] != "P")
    u0 = synth.random_velocity(n, bc, 81)
    ou = oracle.project(g, *u0, dt_over_rho0=0.5)
    plan = vp.Plan(n, g.widths[0][0], g.widths[1][0], dz, bc)
    u = [dev(a) for a in u0]
    p = plan.project(*u, dt_over_rho0=0.5)
    assert rel(host(p), ou[3]) < TOL
    for a in range(3):
        assert rel(host(u[a]), ou[a]) < TOL
    C, _ = synth.droplet(n, bc, 82, dz=dz)
    mdot = np.ones(g.shape)
    ref = oracle.extend_liquid_velocity(g, *ou[:3], C, mdot, 100.0, 1.0)
    out = plan.extend(*u, dev(C), dev(mdot), 100.0, 1.0)
    for a in range(7):
        assert rel(host(out[a]), ref[a]) < TOL, a
    plan.close()
