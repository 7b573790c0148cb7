"""Thin Python binding of the vofp C ABI (``include/vofp.h``): argument marshalling only.

Every function keeps the C name and passes device pointers (``tensor.data_ptr()``) and the current CUDA
stream to the library; all arithmetic of the solve runs in the library's kernels.  Importing this module
fails loudly if the library has not been built (``python -m paper_1907_00890_gb300.build``); there is no
CPU fallback.  With ``VOFP_CHECKED=1`` in the environment it loads the bounds-checked library instead.
"""
import ctypes
import os

import numpy as np

from .build import lib_path

BC = {"P": 0, "NN": 1, "DD": 2, "ND": 3, "DN": 4}
FP64, MIXED, FF = 0, 1, 2

CHECKED = os.environ.get("VOFP_CHECKED", "0") == "1"
LIB = lib_path(CHECKED)
if not os.path.exists(LIB):
    raise ImportError("vofp library not built: %s is missing (run paper_1907_00890_gb300.build.build(%s))"
                      % (LIB, "checked=True" if CHECKED else ""))
_lib = ctypes.CDLL(LIB)


class vofp_opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("tol", ctypes.c_double), ("max_refine", ctypes.c_int),
                ("grad_mode", ctypes.c_int), ("tune", ctypes.c_int)]


class vofp_info(ctypes.Structure):
    _fields_ = [("compat_defect", ctypes.c_double), ("mean_removed", ctypes.c_double),
                ("rel_residual", ctypes.c_double), ("err_estimate", ctypes.c_double),
                ("refine_iters", ctypes.c_int), ("status", ctypes.c_int)]


_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_lib.vofp_opts_default.argtypes = [ctypes.POINTER(vofp_opts)]
_lib.vofp_opts_default.restype = None
_lib.vofp_plan_create.argtypes = [_I, _I, _I, _D, _D, ctypes.POINTER(_D), ctypes.POINTER(_I),
                                  ctypes.POINTER(vofp_opts), ctypes.POINTER(_P)]
_lib.vofp_plan_create.restype = _I
_lib.vofp_plan_destroy.argtypes = [_P]
_lib.vofp_plan_destroy.restype = None
_lib.vofp_plan_workspace_bytes.argtypes = [_P]
_lib.vofp_plan_workspace_bytes.restype = ctypes.c_size_t
_lib.vofp_poisson_solve.argtypes = [_P, _P, _P, _P, ctypes.POINTER(vofp_info)]
_lib.vofp_poisson_solve.restype = _I
_lib.vofp_project.argtypes = [_P, _P, _P, _P, _P, _D, _P, _P, ctypes.POINTER(vofp_info)]
_lib.vofp_project.restype = _I
_lib.vofp_extend_liquid_velocity.argtypes = [_P, _P, _P, _P, _P, _P, _D, _D, _P, _P, _P, _P, _P, _P, _P, _P,
                                             ctypes.POINTER(vofp_info)]
_lib.vofp_extend_liquid_velocity.restype = _I
_lib.vofp_extend_vapour_velocity.argtypes = [_P, _P, _P, _P, _P, _P, _D, _D, _P, _P, _P, _P, _P, _P, _P, _P,
                                             ctypes.POINTER(vofp_info)]
_lib.vofp_extend_vapour_velocity.restype = _I
_lib.vofp_stefan_source.argtypes = [_P, _P, _P, _D, _D, _P, _P]
_lib.vofp_stefan_source.restype = _I
_lib.vofp_project_stefan.argtypes = [_P, _P, _P, _P, _P, _P, _D, _D, _D, _P, _P, ctypes.POINTER(vofp_info)]
_lib.vofp_project_stefan.restype = _I
_lib.vofp_project_vd.argtypes = [_P, _P, _P, _P, _P, _P, _P, _P, _D, _D, _D, _D, _P, _P, ctypes.POINTER(vofp_info)]
_lib.vofp_project_vd.restype = _I
_lib.vofp_vof_update.argtypes = [_P, _P, _P, _P, _P, _D, _P, _P, _P]
_lib.vofp_vof_update.restype = _I
_lib.vofp_trace_enable.argtypes = [_I]
_lib.vofp_trace_enable.restype = _I
_lib.vofp_trace_collect.argtypes = [ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_ulonglong), _I]
_lib.vofp_trace_collect.restype = _I
_lib.vofp_trace_kernel_classes.argtypes = []
_lib.vofp_trace_kernel_classes.restype = _I
_lib.vofp_trace_name.argtypes = [_I]
_lib.vofp_trace_name.restype = ctypes.c_char_p
_lib.vofp_launch_count.argtypes = []
_lib.vofp_launch_count.restype = ctypes.c_ulonglong
_lib.vofp_debug_fail_alloc.argtypes = [ctypes.c_longlong]
_lib.vofp_debug_fail_alloc.restype = _I
_lib.vofp_error_string.argtypes = [_I]
_lib.vofp_error_string.restype = ctypes.c_char_p

EXPORTED = ["vofp_opts_default", "vofp_plan_create", "vofp_plan_destroy", "vofp_plan_workspace_bytes",
            "vofp_poisson_solve", "vofp_project", "vofp_extend_liquid_velocity", "vofp_error_string",
            "vofp_stefan_source", "vofp_project_stefan", "vofp_launch_count", "vofp_trace_enable",
            "vofp_trace_collect", "vofp_trace_kernel_classes", "vofp_trace_name", "vofp_debug_fail_alloc"]


def vofp_debug_fail_alloc(after):
    """Make the (after + 1)-th next device / pinned allocation of the library fail once (after < 0: off)."""
    return _lib.vofp_debug_fail_alloc(int(after))


_lib.vofp_debug_check_word.argtypes = [ctypes.POINTER(ctypes.c_longlong), _I]
_lib.vofp_debug_check_word.restype = _I
_lib.vofp_debug_check_selftest.argtypes = [_P]
_lib.vofp_debug_check_selftest.restype = _I
EXPORTED += ["vofp_debug_check_word", "vofp_debug_check_selftest"]


def vofp_debug_check_word(reset=False):
    """Bounds-checked library: (status, {count, site, index, extent}) of the failed index tests so far, summed
    over the library's translation units (status 1; the plain library returns 0 and zeros)."""
    w = (ctypes.c_longlong * 4)()
    st = _lib.vofp_debug_check_word(w, 1 if reset else 0)
    return st, {"count": w[0], "site": w[1], "index": w[2], "extent": w[3]}


def vofp_debug_check_selftest():
    """One index test that fails by construction (no memory access), on the current stream."""
    import torch
    return _lib.vofp_debug_check_selftest(_P(torch.cuda.current_stream().cuda_stream))


_lib.vofp_project_extend.argtypes = [_P, _P, _P, _P, _P, _P, _D, _D, _D, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                     ctypes.POINTER(vofp_info)]
_lib.vofp_project_extend.restype = _I
EXPORTED.append("vofp_project_extend")


_lib.vofp_project_extend_host.argtypes = [_P, _P, _P, _P, _P, _P, _D, _D, _D, _P, _P, _P, _P, _P, _P, _P, _P]
_lib.vofp_project_extend_host.restype = _I
EXPORTED.append("vofp_project_extend_host")


def vofp_project_extend_host(plan, u, v, w, C, mdot, rho1, rho2, dt_over_rho0, u_out, v_out, w_out, p_out,
                             ug, vg, wg, stream=None):
    """The droplet step on host (CPU) tensors: copies in, both solves, copies out, overlapped on the device.
    Asynchronous on `stream` (default: the current stream); the tensors must stay alive until it completes."""
    def hp(t, name):
        if t is None or t.device.type != "cpu" or t.dtype.itemsize != 8 or not t.is_contiguous():
            raise ValueError("%s: a contiguous float64 CPU tensor is required" % name)
        return t.data_ptr()
    return _check(_lib.vofp_project_extend_host(
        plan, hp(u, "u"), hp(v, "v"), hp(w, "w"), hp(C, "C"), hp(mdot, "mdot"), float(rho1), float(rho2),
        float(dt_over_rho0), hp(u_out, "u_out"), hp(v_out, "v_out"), hp(w_out, "w_out"), hp(p_out, "p_out"),
        hp(ug, "ug"), hp(vg, "vg"), hp(wg, "wg"), _stream(stream)), "vofp_project_extend_host")


def vofp_project_extend(plan, u, v, w, C, mdot, rho1, rho2, dt_over_rho0, p, ue, ve, we, ug=None, vg=None,
                        wg=None, phi=None, stream=None, info=False):
    inf = vofp_info() if info else None
    s = _check(_lib.vofp_project_extend(
        plan, _ptr(u, name="u"), _ptr(v, name="v"), _ptr(w, name="w"), _ptr(C, name="C"), _ptr(mdot, name="mdot"),
        float(rho1), float(rho2), float(dt_over_rho0), _ptr(p, name="p"), _ptr(ue, name="ue"), _ptr(ve, name="ve"),
        _ptr(we, name="we"), _ptr(ug, name="ug"), _ptr(vg, name="vg"), _ptr(wg, name="wg"), _ptr(phi, name="phi"),
        _stream(stream), ctypes.byref(inf) if info else None), "vofp_project_extend")
    return (s, _info_dict(inf)) if info else s


class vofp_request(ctypes.Structure):
    _fields_ = [("n", _I * 3), ("dx", _D), ("dy", _D), ("dz", ctypes.POINTER(_D)), ("bc", _I * 3),
                ("u", _P), ("v", _P), ("w", _P), ("src", _P), ("dt_over_rho0", _D), ("p", _P),
                ("arrival_s", _D)]


_ULL = ctypes.c_ulonglong
_lib.vofp_server_create.argtypes = [ctypes.c_size_t, _I, ctypes.POINTER(vofp_opts), ctypes.POINTER(_P)]
_lib.vofp_server_create.restype = _I
_lib.vofp_server_submit.argtypes = [_P, ctypes.POINTER(vofp_request), ctypes.POINTER(_ULL)]
_lib.vofp_server_submit.restype = _I
_lib.vofp_server_poll.argtypes = [_P, _ULL, ctypes.POINTER(vofp_info), ctypes.POINTER(_D)]
_lib.vofp_server_poll.restype = _I
_lib.vofp_server_wait.argtypes = [_P, _ULL, _D, ctypes.POINTER(vofp_info), ctypes.POINTER(_D)]
_lib.vofp_server_wait.restype = _I
_lib.vofp_server_stats.argtypes = [_P, ctypes.POINTER(_D), _I, _I]
_lib.vofp_server_stats.restype = _I
_lib.vofp_server_destroy.argtypes = [_P]
_lib.vofp_server_destroy.restype = None
_lib.vofp_server_clock.argtypes = [_P, ctypes.POINTER(_D)]
_lib.vofp_server_clock.restype = _I
EXPORTED += ["vofp_server_create", "vofp_server_submit", "vofp_server_poll", "vofp_server_wait",
             "vofp_server_stats", "vofp_server_destroy", "vofp_server_clock"]
SERVER_STATS = 19


def vofp_server_create(mem_budget_bytes=0, max_inflight=16, opts=None):
    h = _P()
    _check(_lib.vofp_server_create(int(mem_budget_bytes), int(max_inflight),
                                   ctypes.byref(opts) if opts is not None else None, ctypes.byref(h)),
           "vofp_server_create")
    return h.value


def vofp_server_submit(server, n, dx, dy, dz, bc, u, v, w, src=None, dt_over_rho0=1.0, p=None, arrival_s=0.0):
    """Submit a projection request; returns its ticket.  The fields must stay valid until it completes.
    ``arrival_s``: when the request arrived, on the server clock (``vofp_server_clock``); 0 = now."""
    dzh = np.ascontiguousarray(np.broadcast_to(np.asarray(dz, dtype=np.float64), (int(n[2]),)))
    r = vofp_request()
    r.n[:] = [int(x) for x in n]
    r.dx, r.dy = float(dx), float(dy)
    r.dz = dzh.ctypes.data_as(ctypes.POINTER(_D))
    r.bc[:] = [BC[b] if isinstance(b, str) else int(b) for b in bc]
    r.u, r.v, r.w = _ptr(u, name="u"), _ptr(v, name="v"), _ptr(w, name="w")
    r.src = _ptr(src, name="src")
    r.dt_over_rho0 = float(dt_over_rho0)
    r.p = _ptr(p, name="p")
    r.arrival_s = float(arrival_s)
    t = _ULL()
    _check(_lib.vofp_server_submit(server, ctypes.byref(r), ctypes.byref(t)), "vofp_server_submit")
    return t.value


def vofp_server_poll(server, ticket):
    """(status, latency_s): status 1 = pending, 0 = done; an error raises."""
    lat = _D()
    s = _lib.vofp_server_poll(server, _ULL(ticket), None, ctypes.byref(lat))
    _check(s, "vofp_server_poll")
    return s, lat.value


def vofp_server_wait(server, ticket, timeout_s=60.0):
    lat = _D()
    _check(_lib.vofp_server_wait(server, _ULL(ticket), float(timeout_s), None, ctypes.byref(lat)),
           "vofp_server_wait")
    return lat.value


def vofp_server_stats(server, reset=False):
    out = (_D * SERVER_STATS)()
    _check(_lib.vofp_server_stats(server, out, SERVER_STATS, 1 if reset else 0), "vofp_server_stats")
    keys = ["completed", "admitted", "rejected", "pending", "arena_in_use", "arena_bytes", "p50_s", "p99_s",
            "cells", "seconds", "worker_prepare_s", "worker_launch_s", "worker_loops", "plan_hits",
            "plan_misses", "plan_evictions", "resident_plans", "p99_wait_submit_s", "p99_wait_queue_s"]
    return dict(zip(keys, list(out)))


def vofp_server_clock(server):
    """Seconds since the server's creation on its own steady clock (the clock of ``arrival_s``)."""
    t = _D()
    _check(_lib.vofp_server_clock(server, ctypes.byref(t)), "vofp_server_clock")
    return t.value


def vofp_server_destroy(server):
    _lib.vofp_server_destroy(server)


_lib.vofp_plan_tune.argtypes = [_P]
_lib.vofp_plan_tune.restype = _I
EXPORTED.append("vofp_plan_tune")


def vofp_plan_tune(plan):
    return _check(_lib.vofp_plan_tune(plan), "vofp_plan_tune")


_lib.vofp_batch_create.argtypes = [ctypes.POINTER(_P), _I, ctypes.POINTER(_P)]
_lib.vofp_batch_create.restype = _I
_lib.vofp_batch_project.argtypes = [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P),
                                    ctypes.POINTER(_P), ctypes.POINTER(_D), ctypes.POINTER(_P), _P]
_lib.vofp_batch_project.restype = _I
_lib.vofp_batch_size.argtypes = [_P]
_lib.vofp_batch_size.restype = _I
_lib.vofp_batch_destroy.argtypes = [_P]
_lib.vofp_batch_destroy.restype = None
EXPORTED += ["vofp_batch_create", "vofp_batch_project", "vofp_batch_size", "vofp_batch_destroy"]


def vofp_batch_create(plans):
    arr = (_P * len(plans))(*plans)
    h = _P()
    _check(_lib.vofp_batch_create(arr, len(plans), ctypes.byref(h)), "vofp_batch_create")
    return h.value


def _ptr_array(ts, name):
    return (_P * len(ts))(*[_ptr(t, name=name) for t in ts])


def vofp_batch_project(batch, u, v, w, src, dt_over_rho0, p, stream=None):
    n = len(u)
    s = _ptr_array(src, "src") if src is not None else None
    pp = _ptr_array(p, "p") if p is not None else None
    dts = (_D * n)(*[float(x) for x in dt_over_rho0])
    return _check(_lib.vofp_batch_project(batch, _ptr_array(u, "u"), _ptr_array(v, "v"), _ptr_array(w, "w"), s,
                                          dts, pp, _stream(stream)), "vofp_batch_project")


def vofp_batch_size(batch):
    return int(_lib.vofp_batch_size(batch))


def vofp_batch_destroy(batch):
    _lib.vofp_batch_destroy(batch)


_lib.vofp_poisson_solve_noalloc.argtypes = [_I, _I, _I, _D, _D, ctypes.POINTER(_D), ctypes.POINTER(_I), _P, _P,
                                            _P]
_lib.vofp_poisson_solve_noalloc.restype = _I
EXPORTED.append("vofp_poisson_solve_noalloc")


def vofp_poisson_solve_noalloc(nx, ny, nz, dx, dy, dz, bc, f, p, stream=None):
    """Allocation-free solve for callers that cannot call cudaMalloc (see include/vofp.h)."""
    dz = np.ascontiguousarray(np.broadcast_to(np.asarray(dz, dtype=np.float64), (int(nz),)))
    codes = (_I * 3)(*[BC[b] if isinstance(b, str) else int(b) for b in bc])
    return _check(_lib.vofp_poisson_solve_noalloc(int(nx), int(ny), int(nz), float(dx), float(dy),
                                                  dz.ctypes.data_as(ctypes.POINTER(_D)), codes,
                                                  _ptr(f, name="f"), _ptr(p, name="p"), _stream(stream)),
                  "vofp_poisson_solve_noalloc")


def vofp_trace_enable(on):
    return int(_lib.vofp_trace_enable(1 if on else 0))


def vofp_trace_kernel_classes():
    return int(_lib.vofp_trace_kernel_classes())


def vofp_trace_name(i):
    return _lib.vofp_trace_name(int(i)).decode()


def vofp_trace_collect():
    """Return {kernel class name: (total ms, launches)} for the traced launches and clear the record."""
    n = vofp_trace_kernel_classes()
    ms = (_D * n)()
    cnt = (ctypes.c_ulonglong * n)()
    _check(_lib.vofp_trace_collect(ms, cnt, n), "vofp_trace_collect")
    return {vofp_trace_name(i): (ms[i], int(cnt[i])) for i in range(n) if cnt[i]}


def vofp_launch_count():
    return int(_lib.vofp_launch_count())


class VofpError(RuntimeError):
    def __init__(self, status, what):
        super().__init__("%s failed: %s (status %d)" % (what, vofp_error_string(status), status))
        self.status = status


def vofp_error_string(status):
    return _lib.vofp_error_string(int(status)).decode()


def _check(status, what):
    if status < 0:
        raise VofpError(status, what)
    return status


def _ptr(t, numel=None, name="array"):
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError("%s must be a contiguous float64 CUDA tensor" % name)
    if numel is not None and t.numel() != numel:
        raise ValueError("%s has %d elements, expected %d" % (name, t.numel(), numel))
    return t.data_ptr()


def _stream(stream):
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def vofp_opts_default():
    o = vofp_opts()
    _lib.vofp_opts_default(ctypes.byref(o))
    return o


def vofp_plan_create(nx, ny, nz, dx, dy, dz, bc, opts=None):
    """Return a plan handle (int).  ``dz``: host array of nz widths; ``bc``: three names or codes."""
    dz = np.ascontiguousarray(np.broadcast_to(np.asarray(dz, dtype=np.float64), (int(nz),)))
    codes = (_I * 3)(*[BC[b] if isinstance(b, str) else int(b) for b in bc])
    h = _P()
    o = ctypes.byref(opts) if opts is not None else None
    _check(_lib.vofp_plan_create(int(nx), int(ny), int(nz), float(dx), float(dy),
                                 dz.ctypes.data_as(ctypes.POINTER(_D)), codes, o, ctypes.byref(h)),
           "vofp_plan_create")
    return h.value


def vofp_plan_destroy(plan):
    _lib.vofp_plan_destroy(plan)


def vofp_plan_workspace_bytes(plan):
    return int(_lib.vofp_plan_workspace_bytes(plan))


def _info_dict(i):
    return {"compat_defect": i.compat_defect, "mean_removed": i.mean_removed, "rel_residual": i.rel_residual,
            "err_estimate": i.err_estimate, "refine_iters": i.refine_iters,
            "status": i.status}


def vofp_poisson_solve(plan, f, p, stream=None, info=False):
    inf = vofp_info() if info else None
    s = _check(_lib.vofp_poisson_solve(plan, _ptr(f, name="f"), _ptr(p, name="p"), _stream(stream),
                                       ctypes.byref(inf) if info else None), "vofp_poisson_solve")
    return (s, _info_dict(inf)) if info else s


def vofp_project(plan, u, v, w, src, dt_over_rho0, p, stream=None, info=False):
    inf = vofp_info() if info else None
    s = _check(_lib.vofp_project(plan, _ptr(u, name="u"), _ptr(v, name="v"), _ptr(w, name="w"),
                                 _ptr(src, name="src"), float(dt_over_rho0), _ptr(p, name="p"), _stream(stream),
                                 ctypes.byref(inf) if info else None), "vofp_project")
    return (s, _info_dict(inf)) if info else s


def vofp_project_vd(plan, u, v, w, src, C, p_n, p_nm1, dt, dt_prev, rho1, rho2, p, stream=None, info=False):
    inf = vofp_info() if info else None
    s = _check(_lib.vofp_project_vd(plan, _ptr(u, name="u"), _ptr(v, name="v"), _ptr(w, name="w"),
                                    _ptr(src, name="src"), _ptr(C, name="C"), _ptr(p_n, name="p_n"),
                                    _ptr(p_nm1, name="p_nm1"), float(dt), float(dt_prev), float(rho1), float(rho2),
                                    _ptr(p, name="p"), _stream(stream), ctypes.byref(inf) if info else None),
               "vofp_project_vd")
    return (s, _info_dict(inf)) if info else s


def vofp_vof_update(plan, C, uG, vG, wG, dt, C_out, work, stream=None):
    return _check(_lib.vofp_vof_update(plan, _ptr(C, name="C"), _ptr(uG, name="uG"), _ptr(vG, name="vG"),
                                       _ptr(wG, name="wG"), float(dt), _ptr(C_out, name="C_out"),
                                       _ptr(work, name="work"), _stream(stream)), "vofp_vof_update")


def vofp_stefan_source(plan, C, mdot, rho1, rho2, s, stream=None):
    return _check(_lib.vofp_stefan_source(plan, _ptr(C, name="C"), _ptr(mdot, name="mdot"), float(rho1),
                                          float(rho2), _ptr(s, name="s"), _stream(stream)), "vofp_stefan_source")


def vofp_project_stefan(plan, u, v, w, C, mdot, rho1, rho2, dt_over_rho0, p, stream=None, info=False):
    inf = vofp_info() if info else None
    s = _check(_lib.vofp_project_stefan(plan, _ptr(u, name="u"), _ptr(v, name="v"), _ptr(w, name="w"),
                                        _ptr(C, name="C"), _ptr(mdot, name="mdot"), float(rho1), float(rho2),
                                        float(dt_over_rho0), _ptr(p, name="p"), _stream(stream),
                                        ctypes.byref(inf) if info else None), "vofp_project_stefan")
    return (s, _info_dict(inf)) if info else s


def vofp_extend_liquid_velocity(plan, u, v, w, C, mdot, rho1, rho2, ue, ve, we, ug=None, vg=None, wg=None,
                                phi=None, stream=None, info=False):
    inf = vofp_info() if info else None
    s = _check(_lib.vofp_extend_liquid_velocity(
        plan, _ptr(u, name="u"), _ptr(v, name="v"), _ptr(w, name="w"), _ptr(C, name="C"),
        _ptr(mdot, name="mdot"), float(rho1), float(rho2), _ptr(ue, name="ue"), _ptr(ve, name="ve"),
        _ptr(we, name="we"), _ptr(ug, name="ug"), _ptr(vg, name="vg"), _ptr(wg, name="wg"), _ptr(phi, name="phi"),
        _stream(stream), ctypes.byref(inf) if info else None), "vofp_extend_liquid_velocity")
    return (s, _info_dict(inf)) if info else s


def vofp_extend_vapour_velocity(plan, u, v, w, C, mdot, rho1, rho2, ue, ve, we, ug=None, vg=None, wg=None,
                                phi=None, stream=None, info=False):
    inf = vofp_info() if info else None
    s = _check(_lib.vofp_extend_vapour_velocity(
        plan, _ptr(u, name="u"), _ptr(v, name="v"), _ptr(w, name="w"), _ptr(C, name="C"),
        _ptr(mdot, name="mdot"), float(rho1), float(rho2), _ptr(ue, name="ue"), _ptr(ve, name="ve"),
        _ptr(we, name="we"), _ptr(ug, name="ug"), _ptr(vg, name="vg"), _ptr(wg, name="wg"), _ptr(phi, name="phi"),
        _stream(stream), ctypes.byref(inf) if info else None), "vofp_extend_vapour_velocity")
    return (s, _info_dict(inf)) if info else s


def face_shapes(n, bc):
    nx, ny, nz = n
    ex = [int((BC[b] if isinstance(b, str) else b) != 0) for b in bc]
    return ((nz, ny, nx + ex[0]), (nz, ny + ex[1], nx), (nz + ex[2], ny, nx))


class Plan:
    """Owns a plan handle; convenience wrappers that allocate outputs with torch (marshalling only)."""

    def __init__(self, n, dx, dy, dz, bc, prec=FP64, tol=1e-10, max_refine=3, grad_mode=0, tune=0):
        o = vofp_opts_default()
        o.prec, o.tol, o.max_refine, o.grad_mode, o.tune = prec, tol, max_refine, grad_mode, tune
        self.n = tuple(int(x) for x in n)
        self.bc = tuple(bc)
        self.handle = vofp_plan_create(self.n[0], self.n[1], self.n[2], dx, dy, dz, bc, o)

    @property
    def cell_shape(self):
        return (self.n[2], self.n[1], self.n[0])

    def face_shapes(self):
        return face_shapes(self.n, self.bc)

    def workspace_bytes(self):
        return vofp_plan_workspace_bytes(self.handle)

    def poisson_solve(self, f, p=None, stream=None, info=False):
        import torch
        if p is None:
            p = torch.empty_like(f)
        r = vofp_poisson_solve(self.handle, f, p, stream, info)
        return (p, r[1]) if info else p

    def project(self, u, v, w, src=None, dt_over_rho0=1.0, p=None, want_p=True, stream=None, info=False):
        import torch
        if p is None and want_p:
            p = torch.empty(self.cell_shape, dtype=torch.float64, device=u.device)
        r = vofp_project(self.handle, u, v, w, src, dt_over_rho0, p, stream, info)
        return (p, r[1]) if info else p

    def project_vd(self, u, v, w, C, p_n, p_nm1, dt, dt_prev, rho1, rho2, src=None, p=None, stream=None,
                   info=False):
        """Variable-density pressure step (u, v, w in place); returns p^{n+1}."""
        import torch
        if p is None:
            p = torch.empty(self.cell_shape, dtype=torch.float64, device=u.device)
        r = vofp_project_vd(self.handle, u, v, w, src, C, p_n, p_nm1, dt, dt_prev, rho1, rho2, p, stream, info)
        return (p, r[1]) if info else p

    def vof_update(self, C, uG, vG, wG, dt, out=None, stream=None):
        """One VoF step with the interface velocity (§3.1); returns C^{n+1} (in `out` if given)."""
        import torch
        if out is None:
            out = torch.empty_like(C)
        work = torch.empty((2,) + tuple(self.cell_shape), dtype=torch.float64, device=C.device)
        vofp_vof_update(self.handle, C, uG, vG, wG, dt, out, work, stream)
        return out

    def stefan_source(self, C, mdot, rho1, rho2, stream=None):
        import torch
        s = torch.empty_like(C)
        vofp_stefan_source(self.handle, C, mdot, rho1, rho2, s, stream)
        return s

    def project_stefan(self, u, v, w, C, mdot, rho1, rho2, dt_over_rho0=1.0, p=None, want_p=True, stream=None,
                       info=False):
        import torch
        if p is None and want_p:
            p = torch.empty(self.cell_shape, dtype=torch.float64, device=u.device)
        r = vofp_project_stefan(self.handle, u, v, w, C, mdot, rho1, rho2, dt_over_rho0, p, stream, info)
        return (p, r[1]) if info else p

    def extend(self, u, v, w, C, mdot, rho1, rho2, want_ug=True, want_phi=True, stream=None, info=False,
               vapour=False):
        """Liquid-velocity extension (§3.6); vapour=True: the boiling variant (Appendix A)."""
        import torch
        ue, ve, we = torch.empty_like(u), torch.empty_like(v), torch.empty_like(w)
        ug = vg = wg = phi = None
        if want_ug:
            ug, vg, wg = torch.empty_like(u), torch.empty_like(v), torch.empty_like(w)
        if want_phi:
            phi = torch.empty(self.cell_shape, dtype=torch.float64, device=u.device)
        fn = vofp_extend_vapour_velocity if vapour else vofp_extend_liquid_velocity
        r = fn(self.handle, u, v, w, C, mdot, rho1, rho2, ue, ve, we, ug, vg, wg, phi, stream, info)
        out = (ue, ve, we, ug, vg, wg, phi)
        return (out, r[1]) if info else out

    def close(self):
        if self.handle:
            vofp_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
