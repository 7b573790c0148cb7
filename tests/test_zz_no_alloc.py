"""The allocation-free Poisson solve against the plan-based one (GPU).

``vofp_poisson_solve_noalloc`` is for callers that cannot call cudaMalloc at solve time (for instance a host
code whose device memory is handed out entirely by its own pool allocator, or a time-stepping loop that must
not pay cudaMalloc's implicit synchronisation): it keeps its workspace in a fixed device array of the
library.  Calls in a row, on different grids up to the array's limits, must each reproduce
``vofp_poisson_solve`` within the FP64 parity tolerance, so nothing left in the shared array by one call
leaks into the next.  This file is
collected last so that a run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

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


def _noalloc(vp, n, dx, dy, dz, bc, f, p):
    import torch
    dzh = np.ascontiguousarray(dz, dtype=np.float64)
    codes = (ctypes.c_int * 3)(*[vp.BC[b] for b in bc])
    fn = vp._lib.vofp_poisson_solve_noalloc
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn(n[0], n[1], n[2], dx, dy, dzh.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), codes,
              f.data_ptr() if f is not None else None, p.data_ptr() if p is not None else None,
              torch.cuda.current_stream().cuda_stream)


def test_noalloc_matches_plan_solve_twice_in_a_row(vp):
    import torch
    # two grids in a row, then the declared limits: odd prime lengths (rolled odd-prime stages, no Bluestein
    # tables in the static array), 1024-cell x and y axes, and the full 2 Mi cells
    cases = [((32, 32, 32), ("P", "P", "NN"), False, 1), ((20, 12, 9), ("DD", "NN", "DN"), True, 2),
             ((31, 13, 10), ("P", "DD", "NN"), True, 3), ((17, 19, 6), ("NN", "P", "P"), False, 4),
             ((1024, 16, 8), ("P", "P", "NN"), True, 5), ((16, 1024, 8), ("NN", "P", "DD"), False, 6),
             ((128, 128, 128), ("P", "P", "NN"), True, 7)]
    for n, bc, stretched, seed in cases:
        dz = synth.stretched_dz(n[2]) if stretched else synth.uniform_dz(n[2])
        dx, dy = 1.0 / n[0], 0.8 / n[1]
        f = torch.tensor(synth.rng(seed).standard_normal((n[2], n[1], n[0])), device="cuda")
        plan = vp.Plan(n, dx, dy, dz, bc)
        ref = plan.poisson_solve(f).cpu().numpy()
        plan.close()
        p = torch.full_like(f, np.nan)
        assert _noalloc(vp, n, dx, dy, dz, bc, f, p) == 0
        torch.cuda.synchronize()
        got = p.cpu().numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < TOL, (n, bc, err)


def test_noalloc_rejects_oversize_before_launch(vp):
    import torch
    f = torch.zeros(1, device="cuda", dtype=torch.float64)
    big = (256, 128, 128)   # 4 Mi cells > 2 Mi cells of static scratch
    assert _noalloc(vp, big, 1.0, 1.0, np.ones(big[2]), ("P", "P", "NN"), f, f) == -8
    long_axis = (2048, 2, 2)
    assert _noalloc(vp, long_axis, 1.0, 1.0, np.ones(2), ("P", "P", "NN"), f, f) == -8
    assert "static scratch" in vp.vofp_error_string(-8)
