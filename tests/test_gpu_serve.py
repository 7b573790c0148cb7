"""GPU tests of the serving loop (continuous batching with memory-based admission).

* requests of uneven sizes submitted back to back with more requests than slots and an arena that holds
  only a few plans at once: every request completes, matches the oracle (mixed: rel-L2 <= 1e-10) and
  matches the same request served alone (to 1e-12: the same kernels run, only FP64 reduction order may
  differ);
* a request whose plan alone exceeds the arena completes with VOFP_ERR_BUSY;
* the latency statistics are filled.
"""
import time

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


def requests(count):
    sizes = synth.serve_sizes(count, lo=16, hi=72)
    out = []
    for i, n in enumerate(sizes):
        bc = ("P", "P", "NN") if i % 3 else ("NN", "DD", "DN")
        dz = synth.stretched_dz(n[2]) if bc[2] != "P" else synth.uniform_dz(n[2])
        out.append(dict(n=n, bc=bc, dz=dz, dx=1.0 / n[0], dy=1.0 / n[1], u0=synth.random_velocity(n, bc, 700 + i),
                        dt=0.5 + 0.1 * i))
    return out


def serve(vp, reqs, budget, inflight):
    import torch
    o = vp.vofp_opts_default()
    o.prec = vp.MIXED
    s = vp.vofp_server_create(budget, inflight, o)
    fields, tickets = [], []
    for r in reqs:
        u = [dev(a) for a in r["u0"]]
        p = torch.empty((r["n"][2], r["n"][1], r["n"][0]), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        tickets.append(vp.vofp_server_submit(s, r["n"], r["dx"], r["dy"], r["dz"], r["bc"], *u,
                                             dt_over_rho0=r["dt"], p=p))
        fields.append((u, p))
    lats = [vp.vofp_server_wait(s, t, 120.0) for t in tickets]
    stats = vp.vofp_server_stats(s)
    vp.vofp_server_destroy(s)
    return fields, lats, stats


def test_served_results_match_oracle_and_alone(vp):
    reqs = requests(12)
    # arena for about three mid-size plans: admission must wait for completions
    budget = 3 * 48 ** 3 * 8 * 4
    fields, lats, stats = serve(vp, reqs, budget, 4)
    assert stats["completed"] == len(reqs) and stats["rejected"] == 0
    assert stats["p99_s"] >= stats["p50_s"] > 0
    assert all(l > 0 for l in lats)
    for r, (u, p) in zip(reqs, fields):
        g = oracle.Grid(*r["n"], r["dx"], r["dy"], r["dz"], r["bc"])
        ou = oracle.project(g, *r["u0"], dt_over_rho0=r["dt"])
        assert rel(p.cpu().numpy(), ou[3]) < TOL
        for a in range(3):
            assert rel(u[a].cpu().numpy(), ou[a]) < TOL
    # the same requests served one at a time
    for idx in (0, 5, 11):
        alone, _, _ = serve(vp, [reqs[idx]], budget, 1)
        assert rel(alone[0][1].cpu().numpy(), fields[idx][1].cpu().numpy()) < 1e-12
        for a in range(3):
            assert rel(alone[0][0][a].cpu().numpy(), fields[idx][0][a].cpu().numpy()) < 1e-12


def test_oversize_request_is_rejected_busy(vp):
    import torch
    o = vp.vofp_opts_default()
    o.prec = vp.MIXED
    s = vp.vofp_server_create(1 << 20, 2, o)   # 1 MiB arena
    n = (64, 64, 64)
    u = [dev(a) for a in synth.random_velocity(n, ("P", "P", "NN"), 3)]
    t = vp.vofp_server_submit(s, n, 1 / 64, 1 / 64, synth.uniform_dz(64), ("P", "P", "NN"), *u)
    with pytest.raises(vp.VofpError) as e:
        vp.vofp_server_wait(s, t, 60.0)
    assert e.value.status == -6
    vp.vofp_server_destroy(s)


@pytest.mark.parametrize("precision", ["mixed", "ff"])
def test_resident_plans_reused_and_evicted(vp, precision):
    """An ensemble of three runs (three grids) submitting in turn: plans stay resident and are reused (three
    new plans for twelve requests); with an arena for about one plan at a time they are evicted instead.
    Every result matches the oracle either way."""
    import torch
    shapes = [((24, 20, 16), ("P", "P", "NN")), ((30, 17, 12), ("NN", "DD", "DN")), ((16, 32, 20), ("P", "P", "NN"))]
    reqs = []
    for i in range(12):
        n, bc = shapes[i % 3]
        dz = synth.stretched_dz(n[2]) if bc[2] != "P" else synth.uniform_dz(n[2])
        reqs.append(dict(n=n, bc=bc, dz=dz, dx=1.0 / n[0], dy=1.0 / n[1],
                         u0=synth.random_velocity(n, bc, 900 + i), dt=1.0))
    o = vp.vofp_opts_default()
    o.prec = vp.MIXED if precision == "mixed" else vp.FF
    o.max_refine = 3 if precision == "mixed" else 0
    sizes = []
    for n, bc in shapes:
        dz = synth.stretched_dz(n[2]) if bc[2] != "P" else synth.uniform_dz(n[2])
        pl = vp.Plan(n, 1.0 / n[0], 1.0 / n[1], dz, bc, prec=o.prec, max_refine=o.max_refine)
        sizes.append(vp.vofp_plan_workspace_bytes(pl.handle) + 256)
        pl.close()
    tight = max(sizes) + min(sizes) // 2  # room for the largest plan, never for two
    for budget, expect_evictions in ((1 << 30, False), (tight, True)):
        s = vp.vofp_server_create(budget, 2, o)
        out = []
        for r in reqs:  # one after another, as a time-stepping ensemble would
            u = [dev(a) for a in r["u0"]]
            p = torch.empty((r["n"][2], r["n"][1], r["n"][0]), dtype=torch.float64, device="cuda")
            t = vp.vofp_server_submit(s, r["n"], r["dx"], r["dy"], r["dz"], r["bc"], *u, dt_over_rho0=r["dt"], p=p)
            vp.vofp_server_wait(s, t, 60.0)
            out.append((u, p))
        st = vp.vofp_server_stats(s)
        vp.vofp_server_destroy(s)
        assert st["completed"] == 12 and st["rejected"] == 0
        if expect_evictions:
            assert st["plan_evictions"] > 0
        else:
            assert st["plan_misses"] == 3 and st["plan_hits"] == 9 and st["plan_evictions"] == 0
        for r, (u, p) in zip(reqs, out):
            g = oracle.Grid(*r["n"], r["dx"], r["dy"], r["dz"], r["bc"])
            ou = oracle.project(g, *r["u0"], dt_over_rho0=r["dt"])
            assert rel(p.cpu().numpy(), ou[3]) < TOL
            for a in range(3):
                assert rel(u[a].cpu().numpy(), ou[a]) < TOL


def test_latency_runs_from_arrival(vp):
    """Latency is charged from the arrival the caller states on the server clock: a request that arrived
    50 ms before it was submitted reports at least 50 ms, and the server's p99 wait before submission shows
    it; an arrival later than the submission counts as the submission."""
    n = (24, 20, 16)
    bc = ("P", "P", "NN")
    o = vp.vofp_opts_default()
    o.prec = vp.FF
    o.max_refine = 0
    s = vp.vofp_server_create(1 << 30, 2, o)
    u = [dev(a) for a in synth.random_velocity(n, bc, 5)]
    time.sleep(0.2)  # the server clock starts at its creation: an arrival 50 ms back must be > 0 on it
    now = vp.vofp_server_clock(s)
    t = vp.vofp_server_submit(s, n, 1.0 / n[0], 1.0 / n[1], synth.uniform_dz(n[2]), bc, *u, arrival_s=now - 0.05)
    lat = vp.vofp_server_wait(s, t, 60.0)
    assert lat >= 0.05
    st = vp.vofp_server_stats(s)
    assert st["p99_wait_submit_s"] >= 0.05 and st["p50_s"] >= 0.05
    t = vp.vofp_server_submit(s, n, 1.0 / n[0], 1.0 / n[1], synth.uniform_dz(n[2]), bc, *u,
                              arrival_s=vp.vofp_server_clock(s) + 10.0)
    assert 0 < vp.vofp_server_wait(s, t, 60.0) < 5.0
    vp.vofp_server_destroy(s)


def test_destroy_with_unpolled_requests_then_fresh_server(vp):
    """A client that submits and never polls (a stalled consumer): destroying the server with requests queued
    and in flight returns once the in-flight work has finished (nothing hangs), and a new server afterwards
    serves a request to oracle parity."""
    import torch
    o = vp.vofp_opts_default()
    o.prec = vp.MIXED
    reqs = requests(24)
    s = vp.vofp_server_create(3 * 48 ** 3 * 8 * 4, 4, o)
    keep = []  # the fields stay valid until destroy has waited for the work on them
    for r in reqs:
        u = [dev(a) for a in r["u0"]]
        torch.cuda.synchronize()
        vp.vofp_server_submit(s, r["n"], r["dx"], r["dy"], r["dz"], r["bc"], *u, dt_over_rho0=r["dt"])
        keep.append(u)
    t0 = time.time()
    vp.vofp_server_destroy(s)
    torch.cuda.synchronize()
    assert time.time() - t0 < 60.0
    del keep
    fields, lats, stats = serve(vp, reqs[:2], 3 * 48 ** 3 * 8 * 4, 2)
    assert stats["completed"] == 2
    for r, (u, p) in zip(reqs[:2], fields):
        g = oracle.Grid(*r["n"], r["dx"], r["dy"], r["dz"], r["bc"])
        ou = oracle.project(g, *r["u0"], dt_over_rho0=r["dt"])
        assert rel(p.cpu().numpy(), ou[3]) < TOL


def test_submit_refuses_malformed_requests_and_keeps_serving(vp):
    """Requests with a non-positive or non-finite step scale, an empty axis or a missing field are refused at
    submission (INVALID_ARG, no ticket); a boundary-condition code out of range is refused when its plan is
    built (the request completes with INVALID_ARG); the server then serves a valid request to parity."""
    import torch
    o = vp.vofp_opts_default()
    o.prec = vp.MIXED
    s = vp.vofp_server_create(64 << 20, 2, o)
    n = (16, 12, 10)
    bc = ("P", "P", "NN")
    dz = synth.uniform_dz(n[2])
    u0 = synth.random_velocity(n, bc, 91)
    u = [dev(a) for a in u0]
    for kw in (dict(dt_over_rho0=0.0), dict(dt_over_rho0=-1.0)):
        with pytest.raises(vp.VofpError) as e:
            vp.vofp_server_submit(s, n, 1 / 16, 1 / 12, dz, bc, *u, **kw)
        assert e.value.status == -1
    with pytest.raises(vp.VofpError) as e:
        vp.vofp_server_submit(s, (16, 0, 10), 1 / 16, 1 / 12, dz, bc, *u)
    assert e.value.status == -1
    with pytest.raises(vp.VofpError) as e:
        vp.vofp_server_submit(s, n, 1 / 16, 1 / 12, dz, bc, u[0], None, u[2])
    assert e.value.status == -1
    t = vp.vofp_server_submit(s, n, 1 / 16, 1 / 12, dz, (0, 0, 7), *u)
    with pytest.raises(vp.VofpError) as e:
        vp.vofp_server_wait(s, t, 60.0)
    assert e.value.status == -1
    u = [dev(a) for a in u0]
    p = torch.empty((n[2], n[1], n[0]), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t = vp.vofp_server_submit(s, n, 1 / 16, 1 / 12, dz, bc, *u, dt_over_rho0=0.7, p=p)
    vp.vofp_server_wait(s, t, 60.0)
    vp.vofp_server_destroy(s)
    g = oracle.Grid(*n, 1 / 16, 1 / 12, dz, bc)
    ou = oracle.project(g, *u0, dt_over_rho0=0.7)
    assert rel(p.cpu().numpy(), ou[3]) < TOL
    for a in range(3):
        assert rel(u[a].cpu().numpy(), ou[a]) < TOL
