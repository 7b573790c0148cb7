"""Benchmark of the projection hot path on synthetic droplet fields.

Workload (one step): the two Poisson solves the VoF solver runs per time step on a 128^3 grid, periodic x, y,
Neumann z, FP64: the pressure projection with the Stefan source of a spherical droplet (radius 0.15 L, tanh
interface 1.5 cells wide, density ratio 100) and the divergence-free liquid-velocity extension that gives the
interface velocity.  Metric: projection Mpts/s = cells x solves / s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--n 128]

Timed region per step: CUDA events on the launching stream around the two library calls, inputs resident
in HBM; L2 is flushed (256 MiB write) and u* restored from a pristine copy before each step, outside the
events.  The roofline's per-kernel launch durations come from a second pass of the same K steps in which
every library launch is bracketed by CUDA events on its own stream (kept out of the first pass, whose
timing the extra events would perturb).  ``e2e`` repeats the measurement through the library's host-buffer call
(vofp_project_extend_host) with pinned host buffers: the H2D copy
of the step's inputs and the D2H copy of its results are inside the timed region.  Under torchrun each rank
runs its own droplet instance (ensemble members are independent: weak scaling, no collective on the data
path); rank 0 prints one JSON line with the max-over-ranks time.  ``--impl reference`` times the CPU oracle
on the host cores instead (rank 0 only).
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the served stream runs up to 64 requests on their own streams: give them as many hardware queues as the
# driver allows (set before the CUDA context exists)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

METRIC = "projection Mpts/s & p99 latency, served/mixed vs plain FP64, rel err ≤1e-10"
UNIT = "Mpts/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed", "ff"],
                    help="arithmetic of the main step (the 128^3 droplet step is specified in FP64)")
    ap.add_argument("--only", choices=["large", "batched", "batched_ff", "served", "vd", "vof"], default=None,
                    help="run one variant alone and print its JSON (for profiling captures); vd: the "
                         "variable-density pressure step on the droplet; vof: the VoF update on the droplet")
    ap.add_argument("--large-n", type=int, default=512,
                    help="cells per axis of the stretched-z projection variant (512 = the specified workload; "
                         "smaller sizes only for profiling captures)")
    ap.add_argument("--large-precisions", default="fp64,mixed,ff",
                    help="precisions of the stretched-z projection variant to run (comma list; one alone for "
                         "profiling captures)")
    ap.add_argument("--tune", action="store_true",
                    help="autotune the stretched-z projection variant's plans (launch shapes, z kernel, radix order)")
    ap.add_argument("--serve-seconds", type=float, default=5.0)
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-sets", type=int, default=8, help="field sets per ensemble run in the served stream")
    ap.add_argument("--no-serve-sweep", dest="serve_sweep", action="store_false",
                    help="skip the served rate sweep")
    ap.add_argument("--record-traffic", metavar="CSV", default=None,
                    help="no GPU: read an ncu launch list (--csv --print-units base, metrics gpu__time_duration.sum, "
                         "dram__bytes_read.sum, dram__bytes_write.sum) and record the DRAM bytes per launch of each "
                         "kernel class in profiles/traffic.json under --traffic-workload, keyed to these sources")
    ap.add_argument("--traffic-workload", default="droplet128_fp64")
    ap.add_argument("--traffic-out", default=os.path.join(ROOT, "profiles", "traffic.json"))
    return ap.parse_args()


def timed_steps(vofp, st, prep, step, steps, trace=True):
    """Mean ms of `steps` steps (CUDA events on stream `st` around each step, `prep` outside them), untraced;
    then, if `trace`, the same steps again with every library launch bracketed by CUDA events on its stream
    (the per-kernel durations of the roofline; kept out of the first pass, whose timing they would perturb).
    Returns (mean ms, per-step ms list, {kernel class: (total ms, launches)} or None)."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        prep()
        ev[i][0].record(st)
        step()
        ev[i][1].record(st)
    torch.cuda.synchronize()
    per = [a.elapsed_time(b) for a, b in ev]
    tr = None
    if trace:
        vofp.vofp_trace_collect()
        vofp.vofp_trace_enable(True)
        for i in range(steps):
            prep()
            step()
        torch.cuda.synchronize()
        vofp.vofp_trace_enable(False)
        tr = vofp.vofp_trace_collect()
    return float(np.mean(per)), per, tr


def bench_mixed_step(vofp, c, u0, C, md, st, flush, args, prec=None, max_refine=3):
    """The same droplet step through a reduced-precision plan (FP32 or FP32-pair transforms + FP64
    low modes, reductions and refinement)."""
    import torch
    prec = vofp.MIXED if prec is None else prec
    plan = vofp.Plan(c["n"], c["dx"], c["dy"], c["dz"], c["bc"], prec=prec, max_refine=max_refine)
    u = [x.clone() for x in u0]
    p = torch.empty(plan.cell_shape, dtype=torch.float64, device=u0[0].device)
    phi = torch.empty_like(p)
    ue = [torch.empty_like(x) for x in u]
    ug = [torch.empty_like(x) for x in u]

    def step():
        vofp.vofp_project_extend(plan.handle, u[0], u[1], u[2], C, md, c["rho1"], c["rho2"], c["dt_over_rho0"], p,
                                 ue[0], ue[1], ue[2], ug[0], ug[1], ug[2], phi)

    def prep():
        for a, b in zip(u, u0):
            a.copy_(b)
        flush.zero_()

    for _ in range(args.warmup):
        prep()
        step()
    torch.cuda.synchronize()
    ms, _, trace = timed_steps(vofp, st, prep, step, args.steps)
    # one more step with info for the refinement statistics
    prep()
    _, info = vofp.vofp_project_extend(plan.handle, u[0], u[1], u[2], C, md, c["rho1"], c["rho2"],
                                       c["dt_over_rho0"], p, ue[0], ue[1], ue[2], ug[0], ug[1], ug[2], phi,
                                       info=True)
    cells = int(np.prod(c["n"]))
    rs = 8 if prec == vofp.FF else 4
    out = {"value": cells * 2 / (ms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": ms,
           "dtype": "f32+f64" if prec == vofp.MIXED else "f32x2+f64", "max_refine": max_refine,
           "refine_iters_both_solves": info["refine_iters"], "rel_residual": info["rel_residual"],
           "per_kernel_ms": {k: round(v[0] / v[1], 5) for k, v in trace.items()},
           "per_step_ms": {k: round(v[0] / args.steps, 5) for k, v in trace.items()},
           "roofline": roofline_mixed(trace, c["n"], rs,
                                      "droplet%d_%s" % (c["n"][0], "mixed" if prec == vofp.MIXED else "ff"))}
    # outputs compared with the oracle's step (ue, ug, phi in the oracle's order) by the caller
    out["_outputs"] = [x.cpu().numpy() for x in ue] + [x.cpu().numpy() for x in ug] + [phi.cpu().numpy()]
    plan.close()
    return out


def bench_vd(vofp, c, u0, C, md, st, flush, args):
    """The variable-density pressure step (Eq. lap_p with its pressure-splitting term) on the same 128^3
    droplet: rho1/rho2 = 100, p^n and p^{n-1} = 0.95 p^n from the seeded pressure-history generator, the
    Stefan source as src, dt = (dt/rho0) rho0 with rho0 = min(rho1, rho2).  One solve per step."""
    import torch
    from paper_1907_00890_gb300 import synth
    plan = vofp.Plan(c["n"], c["dx"], c["dy"], c["dz"], c["bc"])
    rho1, rho2 = c["rho1"], c["rho2"]
    dt = c["dt_over_rho0"] * min(rho1, rho2)
    src = plan.stefan_source(C, md, rho1, rho2)
    pn_h, pm_h = synth.pressure_history(c["C"], synth.BASE_SEED + 7)
    pn = torch.tensor(pn_h, dtype=torch.float64, device=C.device)
    pm = torch.tensor(pm_h, dtype=torch.float64, device=C.device)
    u = [x.clone() for x in u0]
    p = torch.empty_like(pn)

    def step():
        vofp.vofp_project_vd(plan.handle, u[0], u[1], u[2], src, C, pn, pm, dt, dt, rho1, rho2, p)

    def prep():
        for a, b in zip(u, u0):
            a.copy_(b)
        flush.zero_()

    for _ in range(args.warmup):
        prep()
        step()
    torch.cuda.synchronize()
    ms, _, trace = timed_steps(vofp, st, prep, step, args.steps)
    prep()
    step()
    torch.cuda.synchronize()
    n = c["n"]
    cells = int(np.prod(n))
    out = {"value": cells / (ms / 1e3) / 1e6, "unit": UNIT, "ms_per_solve": ms,
           "per_kernel_ms": {k: round(v[0] / v[1], 5) for k, v in trace.items()},
           "workload": "variable-density pressure step %d^3, rho1/rho2 = %g, p^n, p^{n-1} given, FP64"
                       % (n[0], rho1 / rho2)}
    if "vd_predict" in trace:
        tot, cnt = trace["vd_predict"]
        by = 72 * cells  # u, v, w read and written (48 B per cell), p^n, p^{n-1}, C read once (24 B)
        hbm, how = peaks()
        gbs = by / (tot / cnt / 1e3) / 1e9
        out["roofline_vd_predict"] = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                                      "frac": gbs / hbm, "bytes_per_cell": 72, "peak_source": how}
    out["_inputs"] = [pn_h, pm_h]  # host arrays from the generator; the oracle computes its own source
    out["_outputs"] = [x.cpu().numpy() for x in u] + [p.cpu().numpy()]
    out["_dt"] = dt
    plan.close()
    return out


def bench_vof(vofp, c, u0, C, md, st, flush, args):
    """The VoF update with the interface velocity (§3.1, Eqs. fluxes and final_corr_2) on the 128^3 droplet:
    uG from the liquid-velocity extension of the droplet's velocity field, dt at a Courant number of 0.5.
    One update per step; the compulsory traffic is C and uG, vG, wG read and C^{n+1} written, 40 B per cell."""
    import torch
    plan = vofp.Plan(c["n"], c["dx"], c["dy"], c["dz"], c["bc"])
    ext = plan.extend(*u0, C, md, c["rho1"], c["rho2"], want_phi=False)
    ug = ext[3:6]
    h = min(c["dx"], c["dy"], float(np.min(c["dz"])))
    dt = 0.5 * h / max(float(x.abs().max()) for x in ug)
    out = torch.empty_like(C)
    work = torch.empty((2,) + tuple(plan.cell_shape), dtype=torch.float64, device=C.device)

    def step():
        vofp.vofp_vof_update(plan.handle, C, ug[0], ug[1], ug[2], dt, out, work, None)

    def prep():
        flush.zero_()

    for _ in range(args.warmup):
        prep()
        step()
    torch.cuda.synchronize()
    ms, _, trace = timed_steps(vofp, st, prep, step, args.steps)
    cells = int(np.prod(c["n"]))
    r = {"value": cells / (ms / 1e3) / 1e6, "unit": UNIT, "ms_per_update": ms, "dt": dt,
         "per_kernel_ms": {k: round(v[0] / v[1], 5) for k, v in trace.items()},
         "workload": "VoF update with the interface velocity, %d^3 droplet, Courant 0.5, FP64" % c["n"][0]}
    if "vof_update" in trace:
        tot, cnt = trace["vof_update"]
        hbm, how = peaks()
        avg_s = tot / cnt / 1e3  # one launch per update (the fused pass)
        gbs = 40 * cells / avg_s / 1e9
        # bound by its FP64 arithmetic (ncu: FP64 pipe 77% busy, DRAM 4%): about 50 flops per cell -- each
        # implicit one-dimensional step 12 (fluxes, velocity difference, division), the correction 14
        gf = VOF_FLOPS_PER_CELL * cells / avg_s / 1e9
        r["roofline_vof_update"] = {"bound": "alu", "achieved": gf, "peak": FP64_NOMINAL_GFLOPS,
                                    "unit": "GFLOP/s", "frac": gf / FP64_NOMINAL_GFLOPS,
                                    "flops_per_cell": VOF_FLOPS_PER_CELL,
                                    "peak_source": "nominal FP64 rate of the recipe",
                                    "other": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                                              "frac": gbs / hbm, "bytes_per_cell": 40, "peak_source": how}}
    plan.close()
    return r


VOF_FLOPS_PER_CELL = 50
# FP64 flops per cell of the refinement path's FP64 passes (their FP32 transforms not counted): the residual's
# 7-point stencil and defect (13), the divergence and its scale (10), the face epilogues as in `algorithmic`
MIXED_FP64_FLOPS = {"residual_update": 13, "x_forward_div": 10, "grad_update": 10, "extend_epilogue": 24,
                    "stefan_source": 20}


def mixed_bytes_per_cell(rs):
    """Algorithmic HBM bytes per cell of each kernel class of the refinement path (rs: bytes per spectrum
    value, 4 for FP32, 8 for FP32 pairs; fields FP64)."""
    return {"x_forward_div": 24 + 8 + rs, "x_forward": 8 + 8 + rs, "residual_update": 8 + 8 + rs,
            "y_forward": 2 * rs, "y_inverse": 2 * rs, "z_tridiag": 2 * rs, "x_inverse": rs + 16,
            "grad_update": 56, "extend_epilogue": 96, "stefan_source": 48}


def roofline_mixed(trace, n, rs=4, workload=None):
    """HBM roofline of the dominant kernel of the refinement path (among the kernel classes that touch every
    cell; the low-mode, gauge and reporting kernels touch a few columns or run once)."""
    per = mixed_bytes_per_cell(rs)
    cand = {k: v for k, v in trace.items() if k in per}
    if not cand:
        return None
    name = max(cand, key=lambda k: cand[k][0])
    tot, cnt = cand[name]
    cells = int(np.prod(n))
    by = per[name] * cells
    hbm, how = peaks()
    gbs = by / (tot / cnt / 1e3) / 1e9
    mem = {"bound": "hbm", "kernel": name, "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
           "launches": cnt, "avg_launch_ms": tot / cnt, "bytes_per_cell": per[name], "peak_source": how,
           "traffic": measured_traffic(workload, name) if workload else None,
           "note": "averages include launches that returned at once after convergence"}
    if name not in MIXED_FP64_FLOPS:
        return mem
    # an FP64 pass: bound by the FP64 pipe (ncu), so its roofline is the FP64 rate, the HBM figure beside it
    gf = MIXED_FP64_FLOPS[name] * cells / (tot / cnt / 1e3) / 1e9
    out = dict(mem, bound="alu", achieved=gf, peak=FP64_NOMINAL_GFLOPS, unit="GFLOP/s",
               frac=gf / FP64_NOMINAL_GFLOPS, flops_per_cell=MIXED_FP64_FLOPS[name],
               peak_source="nominal FP64 rate of the recipe")
    out.pop("bytes_per_cell")
    out["other"] = {k: mem[k] for k in ("bound", "achieved", "peak", "unit", "frac", "bytes_per_cell", "peak_source")}
    return out


def _torch_laplacian_ppnn(torch, p, dx, dy, dz):
    """The MAC 7-point operator L p for periodic x, y and Neumann z ends (ghost = p), in plain PyTorch FP64:
    the manufactured right-hand sides of the error statements below (no library kernel involved)."""
    lx = (torch.roll(p, -1, 2) - 2.0 * p + torch.roll(p, 1, 2)) / (dx * dx)
    ly = (torch.roll(p, -1, 1) - 2.0 * p + torch.roll(p, 1, 1)) / (dy * dy)
    dzt = torch.tensor(dz, dtype=torch.float64, device=p.device)
    h = 0.5 * (dzt[1:] + dzt[:-1])                      # centre distances across interior z faces
    flux = (p[1:] - p[:-1]) / h[:, None, None]           # interior z faces; the two N end faces carry 0
    lz = torch.zeros_like(p)
    lz[:-1] += flux
    lz[1:] -= flux
    lz /= dzt[:, None, None]
    return lx + ly + lz


def bench_large(vofp, args):
    """512^3 pressure projection, stretched z (tanh clustering, ratio 1.05), P,P,NN, random face velocities:
    refinement path (FP32 transforms + FP64 low modes / reductions / defect correction), FP32 pairs with one
    confirming correction, and the plain FP64 path.  Each result's error is stated against exact solutions of
    the same discrete system: p* smooth (low modes, where a direct solve's eps * cond error sits) and p*
    white noise, f = L p* by a plain PyTorch FP64 stencil; beside them the library's own a-posteriori
    estimate for the projection (info.err_estimate) and its FP64 residual."""
    import torch
    from paper_1907_00890_gb300 import synth
    n = (args.large_n,) * 3
    bc = ("P", "P", "NN")
    dz = synth.stretched_dz(n[2])
    dx = dy = 1.0 / n[0]
    gen = torch.Generator(device="cuda")
    gen.manual_seed(synth.BASE_SEED + 7)
    fs = synth.face_shapes(n, bc)
    u0 = [torch.randn(s, generator=gen, dtype=torch.float64, device="cuda") for s in fs]
    u0[2][0].zero_()
    u0[2][-1].zero_()
    u = [x.clone() for x in u0]
    p = torch.empty(n[::-1], dtype=torch.float64, device="cuda")
    # manufactured exact solutions (zero volume-weighted mean, the solver's gauge)
    dzt = torch.tensor(dz, dtype=torch.float64, device="cuda")
    zc = torch.cumsum(dzt, 0) - 0.5 * dzt
    xc = (torch.arange(n[0], dtype=torch.float64, device="cuda") + 0.5) * dx
    yc = (torch.arange(n[1], dtype=torch.float64, device="cuda") + 0.5) * dy
    smooth = (torch.cos(2 * math.pi * xc)[None, None, :] * torch.sin(2 * math.pi * yc)[None, :, None]
              * torch.cos(math.pi * zc)[:, None, None] + 0.5 * torch.cos(math.pi * zc)[:, None, None]
              + 0.25 * torch.sin(4 * math.pi * xc)[None, None, :] * torch.cos(2 * math.pi * zc)[:, None, None])
    white = torch.randn(n[::-1], generator=gen, dtype=torch.float64, device="cuda")
    vol = dzt[:, None, None].expand(n[::-1])
    exact = {}
    for name, ps in (("smooth", smooth), ("white", white)):
        ps -= (ps * vol).sum() / vol.sum()
        exact[name] = (ps, _torch_laplacian_ppnn(torch, ps, dx, dy, dz))
    del smooth, white, vol
    out = {"workload": "pressure projection %d^3, stretched z (tanh, ratio 1.05), P,P,NN, N(0,1) face velocities; "
                       "one solve per call, inputs > L2" % n[0],
           "error_statement": "rel. L2 error of p against exact solutions p* of the same discrete system (smooth "
                              "low-mode p* and white-noise p*, f = L p* by a plain PyTorch FP64 stencil); "
                              "err_estimate: the library's a-posteriori estimate for the projection"}
    reps = max(3, min(args.steps, 8))
    for name, prec, mr in (("fp64", vofp.FP64, 1), ("mixed", vofp.MIXED, 3), ("ff", vofp.FF, 1)):
        if name not in getattr(args, "large_precisions", "fp64,mixed,ff").split(","):
            continue
        plan = vofp.Plan(n, dx, dy, dz, bc, prec=prec, max_refine=mr, tune=1 if args.tune else 0)
        st = torch.cuda.current_stream()

        def call(info=False):
            return vofp.vofp_project(plan.handle, u[0], u[1], u[2], None, 1.0, p, info=info)

        for _ in range(2):
            for a, b in zip(u, u0):
                a.copy_(b)
            call()
        torch.cuda.synchronize()

        def prep():
            for a, b in zip(u, u0):
                a.copy_(b)

        ms, _, trace = timed_steps(vofp, st, prep, call, reps)
        for a, b in zip(u, u0):
            a.copy_(b)
        _, info = call(info=True)
        cells = int(np.prod(n))
        r = {"value": cells / (ms / 1e3) / 1e6, "unit": UNIT, "ms_per_solve": ms, "solves_per_s": 1e3 / ms,
             "rel_residual": info["rel_residual"], "refine_iters": info["refine_iters"],
             "err_estimate": info["err_estimate"], "max_refine": mr,
             "per_step_ms": {k: round(v[0] / reps, 4) for k, v in trace.items()}}
        for ename, (ps, fs_) in exact.items():
            plan.poisson_solve(fs_, p)
            nps = torch.linalg.vector_norm(ps)
            d = p - ps
            r["rel_err_vs_exact_" + ename] = float(torch.linalg.vector_norm(d) / nps)
            # the part of that error that is a constant offset (the gauge), relative like the error
            off = (d * dzt[:, None, None]).sum() / (dzt.sum() * n[0] * n[1])
            r["gauge_offset_" + ename] = float(off.abs() * math.sqrt(d.numel()) / nps)
            del d
        if prec == vofp.FP64:
            r["dtype"] = "f64"
            r["roofline"] = roofline_from_trace(trace, n, "projection512_fp64")
        else:
            r["dtype"] = "f32+f64" if prec == vofp.MIXED else "f32x2+f64"
            r["roofline"] = roofline_mixed(trace, n, 8 if prec == vofp.FF else 4, "projection512_" + name)
        out[name] = r
        plan.close()
        torch.cuda.empty_cache()
    del u, u0, p, exact
    torch.cuda.empty_cache()
    return out


def bench_batched(vofp, args, prec=None, fp64_baseline=False):
    """64 independent instances, per-axis sizes from {32,48,64,96,128,160}, one graph replay per step."""
    import torch
    from paper_1907_00890_gb300 import synth
    prec = vofp.MIXED if prec is None else prec
    sizes = synth.batch_sizes(64)
    bc = ("P", "P", "NN")
    plans, us = [], []
    gen = torch.Generator(device="cuda")
    gen.manual_seed(synth.BASE_SEED + 4)
    for n in sizes:
        plans.append(vofp.Plan(n, 1.0 / n[0], 1.0 / n[1], synth.uniform_dz(n[2]), bc, prec=prec,
                               max_refine=0 if prec == vofp.FF else 3))
        us.append([torch.randn(s, generator=gen, dtype=torch.float64, device="cuda")
                   for s in synth.face_shapes(n, bc)])
        for a in us[-1][2:]:
            a[0].zero_()
            a[-1].zero_()
    u0 = [[x.clone() for x in u] for u in us]
    b = vofp.vofp_batch_create([p.handle for p in plans])
    dts = [1.0] * len(plans)
    cells = sum(int(np.prod(n)) for n in sizes)

    def prep():
        for u, v in zip(us, u0):
            for a, bb in zip(u, v):
                a.copy_(bb)

    for _ in range(max(2, args.warmup)):
        prep()
        vofp.vofp_batch_project(b, [u[0] for u in us], [u[1] for u in us], [u[2] for u in us], None, dts, None)
    torch.cuda.synchronize()
    reps = max(3, min(args.steps, 10))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    st = torch.cuda.current_stream()
    for i in range(reps):
        prep()
        ev[i][0].record(st)
        vofp.vofp_batch_project(b, [u[0] for u in us], [u[1] for u in us], [u[2] for u in us], None, dts, None)
        ev[i][1].record(st)
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(bb) for a, bb in ev]))
    # accuracy: one instance against its own plan-based single solve is covered by the tests; here the
    # divergence left in every instance (FP64 stencil on the device) relative to the input's
    worst = 0.0
    for p, u, v in zip(plans, us, u0):
        worst = max(worst, _div_ratio(torch, p, u, v))
    vofp.vofp_batch_destroy(b)
    for p in plans:
        p.close()
    # the plain FP64 path on the same ensemble, one projection call per instance (same inputs, same stream)
    ms64 = None
    if fp64_baseline:
        plans64 = [vofp.Plan(n, 1.0 / n[0], 1.0 / n[1], synth.uniform_dz(n[2]), bc) for n in sizes]

        def all64():
            for pl, u in zip(plans64, us):
                vofp.vofp_project(pl.handle, u[0], u[1], u[2], None, 1.0, None)

        prep()
        all64()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for i in range(reps):
            prep()
            ev[i][0].record(st)
            all64()
            ev[i][1].record(st)
        torch.cuda.synchronize()
        ms64 = float(np.mean([a.elapsed_time(bb) for a, bb in ev]))
        for pl in plans64:
            pl.close()
    return {"value": cells / (ms / 1e3) / 1e6, "unit": UNIT, "ms_per_batch": ms, "instances": len(sizes),
            "cells": cells, "solves_per_s": len(sizes) / (ms / 1e3),
            "fp64_one_call_per_instance": None if ms64 is None else {
                "ms": ms64, "solves_per_s": len(sizes) / (ms64 / 1e3), "value": cells / (ms64 / 1e3) / 1e6},
            "dtype": "f32+f64" if prec == vofp.MIXED else "f32x2+f64",
            "max_rel_divergence_after": worst,
            "workload": "64 projection instances, sizes per axis from {32,48,64,96,128,160}, P,P,NN, %s, "
                        "one CUDA-graph replay per batch" % ("FP32 + refinement" if prec == vofp.MIXED
                                                             else "FP32-pair transforms")}


def _div_ratio(torch, plan, u, u0):
    """max |D u| / max |D u0| on the device (MAC divergence, FP64; u: projected faces, u0: the input)."""
    nx, ny, nz = plan.n

    def div(f):
        a, b, c = f
        dx = 1.0 / nx
        d = (a[:, :, 1:] - a[:, :, :-1]) / dx if a.shape[2] == nx + 1 else (torch.roll(a, -1, 2) - a) / dx
        d = d + ((b[:, 1:, :] - b[:, :-1, :]) * ny if b.shape[1] == ny + 1 else (torch.roll(b, -1, 1) - b) * ny)
        d = d + (c[1:] - c[:-1]) * nz
        return d.abs().max().item()

    return div(u) / max(div(u0), 1e-300)


def _serve_stream(vofp, torch, prec, max_refine, rate, warm, dur, runs, bufs, seed):
    """One server fed a Poisson arrival stream: every request belongs to one of the ensemble's runs and uses
    one of that run's field sets; a request whose run has no free set waits on the client side (its latency
    still counts from its arrival, passed to the server as arrival_s)."""
    from paper_1907_00890_gb300 import synth
    rng = synth.rng(seed)
    nreq = int((warm + dur) * rate * 1.2) + 16
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=nreq))
    arrivals = arrivals[arrivals < warm + dur]
    pick = rng.integers(0, len(runs), size=len(arrivals))
    bc = ("P", "P", "NN")
    o = vofp.vofp_opts_default()
    o.prec = prec
    o.max_refine = max_refine
    s = vofp.vofp_server_create(0, 64, o)
    free = [list(range(len(bufs[k]))) for k in range(len(runs))]
    busy = {}
    waiting = []
    t_srv0 = vofp.vofp_server_clock(s)
    t0 = time.perf_counter()
    reset_done = False
    i = 0
    late = 0
    offered = 0
    while i < len(arrivals) or busy or waiting:
        now = time.perf_counter() - t0
        if not reset_done and now >= warm:
            vofp.vofp_server_stats(s, reset=True)
            reset_done = True
        for t in list(busy):
            st_, _ = vofp.vofp_server_poll(s, t)
            if st_ == 0:
                k, b = busy.pop(t)
                free[k].append(b)
        while i < len(arrivals) and arrivals[i] <= now:
            waiting.append(i)
            offered += arrivals[i] >= warm
            i += 1
        still = []
        for j in waiting:
            k = int(pick[j])
            if not free[k]:
                still.append(j)
                continue
            b = free[k].pop()
            n = runs[k]
            t = vofp.vofp_server_submit(s, n, 1.0 / n[0], 1.0 / n[1], synth.uniform_dz(n[2]), bc, *bufs[k][b],
                                        arrival_s=t_srv0 + arrivals[j])
            busy[t] = (k, b)
            if now - arrivals[j] > 0.01:
                late += 1
        waiting = still
        if now > warm + dur + 60.0:
            break
        time.sleep(0.0001)
    st = vofp.vofp_server_stats(s)
    vofp.vofp_server_destroy(s)
    return {"offered_per_s": offered / dur, "solves_per_s": st["completed"] / st["seconds"],
            "p50_ms": st["p50_s"] * 1e3, "p99_ms": st["p99_s"] * 1e3,
            "p99_wait_before_submit_ms": st["p99_wait_submit_s"] * 1e3,
            "p99_wait_in_queue_ms": st["p99_wait_queue_s"] * 1e3,
            "value": st["cells"] / st["seconds"] / 1e6, "unit": UNIT, "completed": int(st["completed"]),
            "rejected": int(st["rejected"]), "late_submissions": late,
            "plan_hits": int(st["plan_hits"]), "plan_misses": int(st["plan_misses"]),
            "plan_evictions": int(st["plan_evictions"]), "resident_plans": int(st["resident_plans"]),
            "worker_prepare_s": round(st["worker_prepare_s"], 3), "worker_launch_s": round(st["worker_launch_s"], 3)}


SERVE_SLO_P99_MS = 100.0


def bench_served(vofp, args):
    """Poisson arrivals of projection requests from an ensemble of 64 droplet runs, each run with its own grid
    (per-axis sizes log-uniform in 48..256, drawn once per run), every request from a run drawn at random;
    served with continuous batching and resident plans: FP32 + refinement, FP32 pairs, and the plain FP64
    path.  Latency runs from each request's scheduled arrival to its completion.  A short sweep then finds
    the highest offered rate each server sustains (completes >= 98% of the offered rate with p99 <= 100 ms)."""
    import torch
    from paper_1907_00890_gb300 import synth
    rate = args.serve_rate
    warm = 1.0
    dur = args.serve_seconds
    runs = synth.serve_sizes(64)
    bc = ("P", "P", "NN")
    # field sets per run at the run's own shape (8 per run, 23 GB in all): a run's requests in flight use
    # distinct sets
    gen = torch.Generator(device="cuda")
    gen.manual_seed(synth.BASE_SEED + 6)
    bufs = [[[torch.randn(fs, generator=gen, dtype=torch.float64, device="cuda") for fs in synth.face_shapes(n, bc)]
             for _ in range(args.serve_sets)] for n in runs]
    servers = (("mixed", vofp.MIXED, 3), ("ff", vofp.FF, 0), ("fp64", vofp.FP64, 1))
    out = {}
    for name, prec, mr in servers:
        r = _serve_stream(vofp, torch, prec, mr, rate, warm, dur, runs, bufs, synth.BASE_SEED + 5)
        r["dtype"] = {vofp.MIXED: "f32+f64", vofp.FF: "f32x2+f64"}.get(prec, "f64")
        r["keeps_up"] = bool(r["solves_per_s"] >= 0.98 * r["offered_per_s"])
        out[name] = r
    if args.serve_sweep:
        sweep = {}
        for name, prec, mr in servers:
            rows = []
            best = 0.0
            for rt in (1000.0, 1500.0, 2000.0, 2500.0, 3000.0, 4000.0):
                r = _serve_stream(vofp, torch, prec, mr, rt, 0.5, 2.0, runs, bufs, synth.BASE_SEED + 50 + int(rt))
                ok = r["solves_per_s"] >= 0.98 * r["offered_per_s"] and r["p99_ms"] <= SERVE_SLO_P99_MS
                rows.append({"rate": rt, "solves_per_s": round(r["solves_per_s"], 1), "p50_ms": round(r["p50_ms"], 2),
                             "p99_ms": round(r["p99_ms"], 2), "sustained": bool(ok)})
                if not ok:
                    break
                best = rt
            sweep[name] = {"max_sustained_req_per_s": best, "rows": rows}
        out["sweep"] = sweep
        out["sweep_rule"] = ("offered rate sustained: >= 98%% of it completed and p99 (arrival -> completion) <= "
                             "%.0f ms, 2 s per rate after 0.5 s warm-up" % SERVE_SLO_P99_MS)
    out["workload"] = ("Poisson arrivals at %.0f req/s for %.0f s after %.0f s warm-up from an ensemble of 64 runs "
                       "(per-axis sizes log-uniform in [48, 256], drawn once per run, %d field sets per run), "
                       "P,P,NN, N(0,1) fields, 64 in flight, resident plans; latency from the scheduled arrival "
                       "to completion" % (rate, dur, warm, args.serve_sets))
    del bufs
    torch.cuda.empty_cache()
    return out


class ClockSampler:
    """Samples SM clock and throttle reasons with nvidia-smi (every 20 ms) while the timed region runs.  The
    device steps of one timed region take some tens of ms and nvidia-smi about a second to start, so the
    sampler is started first (``wait_first``) and kept running over the timed, the traced and the end-to-end
    steps; ``summary(t0, t1)`` keeps the samples read between t0 and t1."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def wait_first(self, timeout=5.0):
        t = time.time()
        while self.proc and not self.lines and time.time() - t < timeout:
            time.sleep(0.01)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0=None, t1=None):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for tl, ln in self.lines:
            if (t0 is not None and tl < t0) or (t1 is not None and tl > t1):
                continue
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) != len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def job_rate(ms_local, cells_per_rank, solves, world, device):
    """Whole-job throughput of replicas: the slowest rank's time (max over ranks) and the cells all ranks
    processed, in Mpts/s.  Returns (max ms, Mpts/s)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, world * cells_per_rank * solves / (ms_max / 1e3) / 1e6


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        if info:
            return int(max(x.get("num_threads", 1) for x in info))
    except Exception:
        pass
    return os.cpu_count() or 1


def oracle_step(c, g):
    import oracle
    ou = oracle.project(g, c["u"], c["v"], c["w"], src=oracle.stefan_source(g, c["C"], c["mdot"], c["rho1"], c["rho2"]),
                        dt_over_rho0=c["dt_over_rho0"])
    return oracle.extend_liquid_velocity(g, *ou[:3], c["C"], c["mdot"], c["rho1"], c["rho2"])


def time_oracle(c, steps, budget_s=20.0):
    """Median seconds per oracle step over at most `steps` steps and about `budget_s` seconds."""
    import oracle
    g = oracle.Grid(*c["n"], c["dx"], c["dy"], c["dz"], c["bc"])
    ts = []
    t_all = time.perf_counter()
    for _ in range(max(1, steps)):
        t0 = time.perf_counter()
        oracle_step(c, g)
        ts.append(time.perf_counter() - t0)
        if time.perf_counter() - t_all > budget_s:
            break
    return float(np.median(ts)), len(ts)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_1907_00890_gb300 import synth
    c = synth.config_droplet(args.n)
    cells = int(np.prod(c["n"]))
    # warm-up, then K timed oracle steps (each the full workload, bounded to a few minutes overall)
    import oracle
    g = oracle.Grid(*c["n"], c["dx"], c["dy"], c["dz"], c["bc"])
    for _ in range(min(args.warmup, 1)):
        oracle_step(c, g)
    ts = []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_step(c, g)
        ts.append(time.perf_counter() - t0)
        if time.perf_counter() - t_all > 150.0:
            break
    sec = float(np.mean(ts))
    value = cells * 2 / sec / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": len(ts),
            "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "droplet step %d^3 (project with Stefan source + liquid-velocity extension), "
                                   "P,P,NN, FP64" % args.n, "grid": list(c["n"]), "solves_per_step": 2},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
                             "sample": "%d full oracle steps of the %d^3 droplet workload" % (len(ts), args.n)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_1907_00890_gb300 import build, synth
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    from paper_1907_00890_gb300 import vofp

    c = synth.config_droplet(args.n, seed_offset=rank)
    n = c["n"]
    cells = int(np.prod(n))
    mixed = args.precision != "fp64"
    prec = {"fp64": vofp.FP64, "mixed": vofp.MIXED, "ff": vofp.FF}[args.precision]
    plan = vofp.Plan(n, c["dx"], c["dy"], c["dz"], c["bc"], prec=prec, max_refine=0 if prec == vofp.FF else 3)
    st = torch.cuda.current_stream()

    def T(a):
        return torch.tensor(a, dtype=torch.float64, device=dev)

    u0 = [T(a) for a in (c["u"], c["v"], c["w"])]
    u = [x.clone() for x in u0]
    C, md = T(c["C"]), T(c["mdot"])
    p = torch.empty(plan.cell_shape, dtype=torch.float64, device=dev)
    phi = torch.empty_like(p)
    ue = [torch.empty_like(x) for x in u]
    ug = [torch.empty_like(x) for x in u]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        vofp.vofp_project_extend(plan.handle, u[0], u[1], u[2], C, md, c["rho1"], c["rho2"], c["dt_over_rho0"], p,
                                 ue[0], ue[1], ue[2], ug[0], ug[1], ug[2], phi)

    def prep():
        for a, b in zip(u, u0):
            a.copy_(b)
        flush.zero_()

    for _ in range(args.warmup):
        prep()
        step()
    torch.cuda.synchronize()

    # ---- device-resident timing ----
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(torch.cuda.current_device()).__enter__()
    clk.wait_first()
    t_clk0 = time.time()
    l0 = vofp.vofp_launch_count()
    for i in range(args.steps):
        prep()
        ev[i][0].record(st)
        step()
        ev[i][1].record(st)
    torch.cuda.synchronize()
    launches = vofp.vofp_launch_count() - l0
    # the same steps once more with per-launch events: kernel durations for the roofline
    _, _, trace = timed_steps(vofp, st, prep, step, args.steps)
    if world > 1:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = float(np.mean(step_ms))
    ms_max, value = job_rate(ms, cells, 2, world, dev)

    # ---- end to end: the same step through the host-buffer call (pinned host memory in and out; the library
    # copies in, solves and copies back, overlapping the transfers with the compute) ----
    h_in = [torch.empty(x.shape, dtype=torch.float64, pin_memory=True) for x in u0 + [C, md]]
    for h, d in zip(h_in, u0 + [C, md]):
        h.copy_(d)
    h_out = [torch.empty(x.shape, dtype=torch.float64, pin_memory=True) for x in u + [p] + ug]
    h2d = sum(x.numel() * 8 for x in h_in)
    d2h = sum(x.numel() * 8 for x in h_out)
    e2e_steps = max(3, min(args.steps, 20))
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(e2e_steps)]

    def host_step():
        vofp.vofp_project_extend_host(plan.handle, h_in[0], h_in[1], h_in[2], h_in[3], h_in[4], c["rho1"],
                                      c["rho2"], c["dt_over_rho0"], h_out[0], h_out[1], h_out[2], h_out[3],
                                      h_out[4], h_out[5], h_out[6])

    for i in range(e2e_steps + 1):
        flush.zero_()
        if i > 0:
            ev2[i - 1][0].record(st)
        host_step()
        if i > 0:
            ev2[i - 1][1].record(st)
    torch.cuda.synchronize()
    t_clk1 = time.time()
    clk.__exit__(None, None, None)
    e2e_ms = float(np.mean([a.elapsed_time(b) for a, b in ev2]))
    _, e2e_value = job_rate(e2e_ms, cells, 2, world, dev)

    # ---- roofline of the dominant kernel (its launches timed with events on the launching stream) ----
    wl = "droplet%d_%s" % (args.n, args.precision)
    roof = roofline_mixed(trace, n, 8 if prec == vofp.FF else 4, wl) if mixed else roofline_from_trace(trace, n, wl)

    # ---- the other forms of the same path: mixed precision, batched ensemble, served stream ----
    variants = {}
    if not args.no_variants:
        variants["mixed_step"] = bench_mixed_step(vofp, c, u0, C, md, st, flush, args)
        variants["ff_step"] = bench_mixed_step(vofp, c, u0, C, md, st, flush, args, prec=vofp.FF, max_refine=0)
        variants["ff_step_confirmed"] = bench_mixed_step(vofp, c, u0, C, md, st, flush, args, prec=vofp.FF)
        variants["variable_density"] = bench_vd(vofp, c, u0, C, md, st, flush, args)
        torch.cuda.empty_cache()
        variants["large_512"] = bench_large(vofp, args)
        torch.cuda.empty_cache()
        variants["batched"] = bench_batched(vofp, args, fp64_baseline=True)
        torch.cuda.empty_cache()
        variants["batched_ff"] = bench_batched(vofp, args, prec=vofp.FF)
        torch.cuda.empty_cache()
        variants["served"] = bench_served(vofp, args)
        torch.cuda.empty_cache()

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": {"fp64": "f64", "mixed": "f32+f64", "ff": "f32x2+f64"}[args.precision],
                "data": "synthetic",
                "config": {"workload": "droplet step %d^3 (project with Stefan source + liquid-velocity extension), "
                                       "P,P,NN, %s" % (args.n, {"fp64": "FP64", "mixed": "mixed precision (FP32 + FP64 refinement)",
                                                               "ff": "FP32-pair transforms"}[args.precision]),
                           "grid": list(n), "solves_per_step": 2,
                           "parallelism": "replicas" if world > 1 else "single",
                           "l2": "flushed between steps (256 MiB write, outside the events)"},
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "gpu_launches": int(launches),
                "clocks": dict(clk.summary(t_clk0, t_clk1), window="timed, traced and end-to-end steps"),
                "roofline": roof}
        if not args.no_cpu_baseline:
            sec, nsteps = time_oracle(c, 10, 20.0)
            line["cpu_baseline"] = {"value": cells * 2 / sec / 1e6, "unit": UNIT, "cores": cpu_threads(),
                                    "kind": "oracle",
                                    "sample": "%d oracle steps (median) of the same %d^3 droplet workload" % (nsteps, args.n)}
            ref = None
            for vk in ("mixed_step", "ff_step", "ff_step_confirmed"):
                if vk not in variants:
                    continue
                # accuracy of the reduced-precision step against the oracle (one step, same inputs)
                if ref is None:
                    import oracle
                    ref = oracle_step(c, oracle.Grid(*c["n"], c["dx"], c["dy"], c["dz"], c["bc"]))
                got = variants[vk].pop("_outputs")
                errs = [float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)) for a, b in zip(got, ref[:7])]
                variants[vk]["max_rel_err_vs_oracle"] = max(errs)
            vd = variants.get("variable_density")
            if vd is not None:
                import oracle
                pn, pm = vd["_inputs"]
                g = oracle.Grid(*c["n"], c["dx"], c["dy"], c["dz"], c["bc"])
                src = oracle.stefan_source(g, c["C"], c["mdot"], c["rho1"], c["rho2"])
                r = oracle.project_variable_density(g, c["u"], c["v"], c["w"], c["C"], pn, pm, vd["_dt"], vd["_dt"],
                                                    c["rho1"], c["rho2"], src=src)
                got = vd["_outputs"]
                vd["max_rel_err_vs_oracle"] = max(
                    float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
                    for a, b in zip(got, (r[0], r[1], r[2], r[3])))
        if variants:
            for vk in ("mixed_step", "ff_step", "ff_step_confirmed", "variable_density"):
                for key in ("_outputs", "_inputs", "_dt"):
                    variants.get(vk, {}).pop(key, None)
            line["variants"] = variants
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()


FP64_NOMINAL_GFLOPS = 1250.0   # GB300 FP64 (vector and tensor), the profiling recipe's unit figure


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def source_sha():
    """Digest of the CUDA sources: DRAM traffic recorded from an ncu capture is valid only for these kernels."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1907_00890_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(d, f), "rb") as fh:
                h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()


def measured_traffic(workload, kernel):
    """DRAM bytes (read + write) per launch of a kernel class, from the ncu summary in profiles/traffic.json,
    or None when that capture was taken on other kernel sources (or is missing)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            t = json.load(fh)
    except Exception:
        return None
    if t.get("source_sha") != source_sha():
        return None
    v = t.get("workloads", {}).get(workload, {}).get(kernel)
    return float(v) if v is not None else None


def algorithmic(kname, n):
    """Algorithmic HBM bytes and FP64 flops of one launch of kernel class ``kname`` on an n-grid.

    Bytes: each compulsory array read or written once (8 B per FP64 value).  Flops: a real-to-real transform
    of length m counts 2.5 m log2 m per line (half the 5 m log2 m of a complex FFT); the z recurrence with
    plan-time factors 6 per point (forward multiply-add and multiply, back multiply-add, output scale);
    stencils their adds and multiplies (a multiply-add counts 2): the velocity correction a difference and a
    multiply-add per face (3, one more product on z faces: 10 per cell), the extension a difference, two face
    sums, a product and two multiply-adds per face (8, 24 per cell), the geometry its three central differences
    and scales, |grad C|^2, the reciprocal square root, s and n (20 per cell).
    """
    nx, ny, nz = n
    cells = nx * ny * nz

    def lg(m):
        return math.log2(m) if m > 1 else 0.0

    tab = {
        "x_forward": (16, 2.5 * lg(nx)),
        "x_forward_div": (32, 8 + 2.5 * lg(nx)),
        "x_forward_stefan": (24, 18 + 2.5 * lg(nx)),
        "x_forward_div_stefan": (48, 26 + 2.5 * lg(nx)),
        "y_forward": (16, 2.5 * lg(ny)),
        "y_inverse": (16, 2.5 * lg(ny)),
        "z_tridiag": (16, 6),
        "x_inverse": (16, 2.5 * lg(nx)),
        "grad_update": (56, 10),
        "extend_epilogue": (96, 24),
        "stefan_source": (48, 20),
    }
    b, f = tab.get(kname, (0, 0))
    return b * cells, f * cells


def roofline_from_trace(trace, n, workload=None):
    """Dominant kernel class (largest summed time) with its achieved rates against the peaks."""
    if not trace:
        return None
    name = max(trace, key=lambda k: trace[k][0])
    tot_ms, cnt = trace[name]
    avg_s = tot_ms / cnt / 1e3
    by, fl = algorithmic(name, n)
    hbm, how = peaks()
    gbs = by / avg_s / 1e9
    gfl = fl / avg_s / 1e9
    share = tot_ms / sum(v[0] for v in trace.values())
    mem = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
           "peak_source": how + " (copy test)"}
    alu = {"bound": "alu", "achieved": gfl, "peak": FP64_NOMINAL_GFLOPS, "unit": "GFLOP/s",
           "frac": gfl / FP64_NOMINAL_GFLOPS, "peak_source": "nominal FP64 rate of the recipe"}
    r = dict(alu if alu["frac"] >= mem["frac"] else mem)
    r.update({"kernel": name, "launches": cnt, "avg_launch_ms": tot_ms / cnt, "share_of_step": share,
              "traffic": measured_traffic(workload, name) if workload else None,
              "other": mem if r["bound"] == "alu" else alu,
              "per_kernel_ms": {k: round(v[0] / v[1], 5) for k, v in trace.items()}})
    return r


def synth_droplet(n):
    from paper_1907_00890_gb300 import synth
    return synth.config_droplet(n)


def run_only(args):
    from paper_1907_00890_gb300 import build
    build.build()
    from paper_1907_00890_gb300 import vofp
    if args.only == "large":
        r = bench_large(vofp, args)
    elif args.only == "batched":
        r = bench_batched(vofp, args)
    elif args.only == "batched_ff":
        r = bench_batched(vofp, args, prec=vofp.FF)
    elif args.only in ("vd", "vof"):
        import torch
        c = synth_droplet(args.n)
        dev = torch.device("cuda", torch.cuda.current_device())
        T = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)  # noqa: E731
        u0 = [T(a) for a in (c["u"], c["v"], c["w"])]
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        fn = bench_vd if args.only == "vd" else bench_vof
        r = fn(vofp, c, u0, T(c["C"]), T(c["mdot"]), torch.cuda.current_stream(), flush, args)
        for key in ("_inputs", "_outputs", "_dt"):
            r.pop(key, None)
    else:
        r = bench_served(vofp, args)
    print(json.dumps({"only": args.only, "result": r}))


# kernel function name (as ncu prints it) -> the library's trace class
_KCLASS = [(r"k_zfactor", None), (r"k_zlow", "z_low_modes"), (r"k_z", "z_tridiag"), (r"k_xinv", "x_inverse"),
           (r"k_xtc\b", "x_tensor_core"), (r"k_grad", "grad_update"), (r"k_extend_epi", "extend_epilogue"),
           (r"k_geometry", "stefan_source"), (r"k_vd_predict", "vd_predict"), (r"k_vof_fused", "vof_update"),
           (r"k_shift", "gauge_shift")]
_XMODE = {0: "x_forward", 1: "x_forward_div", 2: "x_forward_stefan", 3: "residual_update", 4: "x_forward_div"}
CLASSES = set(c for _, c in _KCLASS) | set(_XMODE.values()) | {"y_forward", "y_inverse"}


def _template_args(name):
    i = name.find("<")
    if i < 0:
        return []
    depth, cur, out = 0, "", []
    for ch in name[i + 1:]:
        if ch == "<":
            depth += 1
        elif ch == ">":
            if depth == 0:
                break
            depth -= 1
        if ch == "," and depth == 0:
            out.append(cur.strip())
            cur = ""
        else:
            cur += ch
    out.append(cur.strip())
    return out


def kernel_class(name):
    """The trace class of a kernel of this library from its (demangled) name; None for others."""
    import re
    ta = [re.sub(r"^\(\w+\)", "", t) for t in _template_args(name)]
    if re.search(r"k_xfwd", name) and ta:
        return _XMODE.get(int(ta[-1])) if ta[-1].isdigit() else None
    if re.search(r"k_ypass", name) and ta:
        inv = ta[1] if "k_ypass_tma" in name else ta[-1]
        return "y_inverse" if inv in ("true", "1") else "y_forward"
    for pat, cls in _KCLASS:
        if re.search(pat, name):
            return cls
    return None


def read_launch_list(path):
    """Per launch (in order): kernel name, class, duration in us, DRAM bytes read + written, from an ncu CSV."""
    import csv
    scale = {"byte": 1.0, "b": 1.0, "kbyte": 1e3, "kb": 1e3, "mbyte": 1e6, "mb": 1e6, "gbyte": 1e9, "gb": 1e9,
             "nsecond": 1e-3, "ns": 1e-3, "usecond": 1.0, "us": 1.0, "msecond": 1e3, "ms": 1e3, "second": 1e6,
             "s": 1e6}
    launches = {}
    with open(path, newline="") as fh:
        rows = [r for r in csv.reader(fh)]
    hdr = next(i for i, r in enumerate(rows) if "Metric Name" in r)
    cols = rows[hdr]
    ci = {c: cols.index(c) for c in ("ID", "Kernel Name", "Metric Name", "Metric Unit", "Metric Value")}
    for r in rows[hdr + 1:]:
        if len(r) < len(cols):
            continue
        lid = int(r[ci["ID"]])
        d = launches.setdefault(lid, {"name": r[ci["Kernel Name"]], "us": 0.0, "bytes": 0.0})
        v = float(r[ci["Metric Value"]].replace(",", "")) * scale.get(r[ci["Metric Unit"]].lower(), 1.0)
        m = r[ci["Metric Name"]]
        if m == "gpu__time_duration.sum":
            d["us"] = v
        elif m in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            d["bytes"] += v
    out = []
    for lid in sorted(launches):
        d = launches[lid]
        out.append(dict(d, cls=kernel_class(d["name"])))
    return out


def record_traffic(args):
    """Write the per-class DRAM bytes per launch of one ncu launch list into profiles/traffic.json (other
    workloads kept only when they were recorded on the same sources) and print the markdown summary table."""
    ls = read_launch_list(args.record_traffic)
    agg = {}
    for d in ls:
        a = agg.setdefault(d["cls"] or d["name"][:40], {"n": 0, "us": 0.0, "bytes": 0.0})
        a["n"] += 1
        a["us"] += d["us"]
        a["bytes"] += d["bytes"]
    path = args.traffic_out
    try:
        with open(path) as fh:
            t = json.load(fh)
    except Exception:
        t = {}
    sha = source_sha()
    if t.get("source_sha") != sha:
        t = {"workloads": {}}
    t["source_sha"] = sha
    t["note"] = ("DRAM bytes (read + write) per launch and kernel class from ncu launch lists of these sources "
                 "(written by bench.py --record-traffic); summaries in profiles/launches_*.md")
    t.setdefault("workloads", {})[args.traffic_workload] = {
        k: round(a["bytes"] / a["n"]) for k, a in sorted(agg.items()) if a["bytes"] > 0 and k in CLASSES}
    with open(path, "w") as fh:
        json.dump(t, fh, indent=1)
        fh.write("\n")
    tot = sum(a["us"] for a in agg.values())
    print("| kernel class | launches | total us | share | DRAM MB / launch |")
    print("|---|---|---|---|---|")
    for k, a in sorted(agg.items(), key=lambda kv: -kv[1]["us"]):
        print("| %s | %d | %.1f | %.3f | %.1f |" % (k, a["n"], a["us"], a["us"] / tot if tot else 0.0,
                                                 a["bytes"] / a["n"] / 1e6))
    print("| total | %d | %.1f | 1.000 | |" % (sum(a["n"] for a in agg.values()), tot))


def main():
    args = parse()
    if args.record_traffic:
        record_traffic(args)
        return
    if args.only:
        run_only(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
