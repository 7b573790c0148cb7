"""Host-side fault injection on the GPU path: out-of-memory at every place the library allocates.

The failure is made on the host (vofp_debug_fail_alloc makes one chosen allocation return an error, as a
fake of the failing cudaMalloc), so no GPU fault is ever caused.  Each call must return VOFP_ERR_OOM
before launching anything, give back what it had already allocated, and the same call must succeed once the
injection is off.  Also: a TMA tile load that never completes is not provoked; its bounded wait is covered by
reading (the kernel records a timeout and returns).
"""
import numpy as np
import pytest

import oracle
from paper_1907_00890_gb300 import synth

pytestmark = pytest.mark.gpu

OOM = -3
SLACK = 4 << 20  # device-memory accounting granularity tolerated when checking for leaks


@pytest.fixture(scope="module")
def vp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_00890_gb300 import build
    build.build()
    from paper_1907_00890_gb300 import vofp
    yield vofp
    vofp.vofp_debug_fail_alloc(-1)


def free_mem():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


N = (24, 20, 16)
BC = ("P", "P", "NN")


def make_plan(vp, prec=0):
    return vp.Plan(N, 1.0 / N[0], 1.0 / N[1], synth.uniform_dz(N[2]), BC, prec=prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_plan_create_out_of_memory(vp, prec):
    pr = 0 if prec == "fp64" else 1
    before = free_mem()
    vp.vofp_debug_fail_alloc(0)
    with pytest.raises(vp.VofpError) as e:
        make_plan(vp, pr)
    assert e.value.status == OOM
    assert abs(free_mem() - before) <= SLACK
    vp.vofp_debug_fail_alloc(-1)
    plan = make_plan(vp, pr)  # the same call succeeds once the injection is off
    plan.close()


def test_extension_geometry_out_of_memory_then_recovers(vp):
    """The interface-geometry block of a plan is allocated on its first extension call: a failure there is
    VOFP_ERR_OOM with nothing launched, and the next call allocates it and matches the oracle."""
    g = oracle.Grid(*N, 1.0 / N[0], 1.0 / N[1], synth.uniform_dz(N[2]), BC)
    C, _ = synth.droplet(N, BC, 4)
    mdot = np.ones(g.shape)
    u0 = synth.random_velocity(N, BC, 6)
    plan = make_plan(vp)
    u = [dev(a) for a in u0]
    launches = vp.vofp_launch_count()
    vp.vofp_debug_fail_alloc(0)
    with pytest.raises(vp.VofpError) as e:
        plan.extend(*u, dev(C), dev(mdot), 100.0, 1.0)
    assert e.value.status == OOM and vp.vofp_launch_count() == launches
    vp.vofp_debug_fail_alloc(-1)
    out = plan.extend(*u, dev(C), dev(mdot), 100.0, 1.0)
    ref = oracle.extend_liquid_velocity(g, *u0, C, mdot, 100.0, 1.0)
    for a in range(3):
        got = out[a].cpu().numpy()
        assert np.linalg.norm(got - ref[a]) <= 1e-12 * np.linalg.norm(ref[a])
    plan.close()


def test_host_step_out_of_memory(vp):
    """The host-buffer step allocates its device fields on first use: a failure there is VOFP_ERR_OOM."""
    import torch
    plan = make_plan(vp)
    fs = vp.face_shapes(N, BC)
    cells = (N[2], N[1], N[0])
    host = lambda s: torch.zeros(s, dtype=torch.float64).pin_memory()  # noqa: E731
    u, v, w = (host(s) for s in fs)
    C, md = host(cells), host(cells)
    uo, vo, wo = (host(s) for s in fs)
    po = host(cells)
    ug, vg, wg = (host(s) for s in fs)
    vp.vofp_debug_fail_alloc(0)
    with pytest.raises(vp.VofpError) as e:
        vp.vofp_project_extend_host(plan.handle, u, v, w, C, md, 100.0, 1.0, 1.0, uo, vo, wo, po, ug, vg, wg)
    assert e.value.status == OOM
    vp.vofp_debug_fail_alloc(-1)
    vp.vofp_project_extend_host(plan.handle, u, v, w, C, md, 100.0, 1.0, 1.0, uo, vo, wo, po, ug, vg, wg)
    torch.cuda.synchronize()
    plan.close()


@pytest.mark.parametrize("which", [0, 1])  # 0: the device argument block, 1: its pinned host staging copy
def test_batch_create_out_of_memory(vp, which):
    plans = [make_plan(vp, 1) for _ in range(3)]
    before = free_mem()
    vp.vofp_debug_fail_alloc(which)
    with pytest.raises(vp.VofpError) as e:
        vp.vofp_batch_create([p.handle for p in plans])
    assert e.value.status == OOM
    assert abs(free_mem() - before) <= SLACK
    vp.vofp_debug_fail_alloc(-1)
    b = vp.vofp_batch_create([p.handle for p in plans])
    vp.vofp_batch_destroy(b)
    for p in plans:
        p.close()


@pytest.mark.parametrize("which", [0, 1, 3])  # 0: the arena; 1, 3: a slot's pinned staging buffer
def test_server_create_out_of_memory(vp, which):
    before = free_mem()
    vp.vofp_debug_fail_alloc(which)
    with pytest.raises(vp.VofpError) as e:
        vp.vofp_server_create(64 << 20, 4)
    assert e.value.status == OOM
    assert abs(free_mem() - before) <= SLACK
    vp.vofp_debug_fail_alloc(-1)
    s = vp.vofp_server_create(64 << 20, 4)
    vp.vofp_server_destroy(s)
