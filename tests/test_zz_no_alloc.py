"""The allocation-free entry point lbmd_lb_step_noalloc, for callers that
cannot allocate device memory (their memory belongs to another framework's
pool, or another thread is capturing a CUDA graph in global mode, or a
real-time loop must not touch the allocator).  It steps caller-owned
populations without a context or workspace, keeping its geometry scratch in a
fixed array inside the library.

Checked against the context path (lbmd_step followed by
lbmd_read_populations) on the same input, for two calls in a row: the second
call must not see anything left over from the first.  Tolerance: 1e-5 relative
per population, the one-step tolerance of the other parity tests."""
import ctypes as C

import numpy as np
import pytest

import seeded_inputs as si

pytestmark = pytest.mark.gpu


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0710_1272_gb300 as lb
    return torch, lb


def _rel(a, b):
    a = a.double()
    b = b.double()
    m = b != 0
    assert bool((a[~m] == 0).all())
    return float(((a[m] - b[m]).abs() / b[m].abs()).max())


@pytest.mark.parametrize("case", [
    dict(nx=48, ny=20, nz=12, wall_x=24, pore_d=4, tau=0.7, body_force=(1e-5, 0.0, 0.0)),
    dict(nx=37, ny=18, nz=9, wall_x=5, wall_thickness=2, pore_d=3, y_walls=1, tau=0.9,
         forcing="guo", body_force=(2e-5, 1e-6, 0.0)),
])
def test_noalloc_step_matches_context_step(case):
    torch, lb = _setup()
    shape = (case["nz"], case["ny"], case["nx"])
    rho, u = si.random_flow(shape, seed=21, u_max=0.04)
    sim = lb.Simulation(case, init_rho=rho, init_u=u)
    cp, keep = lb.make_params(case)
    stream = sim.stream.cuda_stream
    f0 = sim.populations_device()
    out = [torch.empty_like(f0), torch.empty_like(f0)]
    src = f0
    for k in range(2):
        lb.lbmd_lb_step_noalloc(cp, src.data_ptr(), out[k].data_ptr(), stream)
        sim.step(1)
        ref = sim.populations_device()
        torch.cuda.synchronize()
        assert _rel(out[k], ref) < 1e-5, k
        src = out[k]
    del keep


def test_noalloc_rejects_boxes_beyond_the_scratch():
    torch, lb = _setup()
    L = lb.load()
    cp, keep = lb.make_params(dict(nx=32, ny=1025, nz=1024, wall_x=-1))
    f = torch.empty(32, dtype=torch.float32, device="cuda")
    g = torch.empty(32, dtype=torch.float32, device="cuda")
    rc = L.lbmd_lb_step_noalloc(C.byref(cp), C.c_void_p(f.data_ptr()), C.c_void_p(g.data_ptr()), None)
    assert rc == lb.lbmd.LBMD_ESIZE
    cp2, keep2 = lb.make_params(dict(nx=8, ny=8, nz=8, wall_x=-1))
    rc = L.lbmd_lb_step_noalloc(C.byref(cp2), C.c_void_p(f.data_ptr()), C.c_void_p(f.data_ptr()), None)
    assert rc == lb.lbmd.LBMD_EINVAL
    # what the entry point does not cover: 16-bit storage, beads, the thermal source
    for bad in (dict(storage="f16"), dict(kT_fluid=1e-4)):
        cp3, keep3 = lb.make_params(dict(nx=8, ny=8, nz=8, wall_x=-1, **bad))
        rc = L.lbmd_lb_step_noalloc(C.byref(cp3), C.c_void_p(f.data_ptr()), C.c_void_p(g.data_ptr()), None)
        assert rc == lb.lbmd.LBMD_EUNSUPPORTED, bad
    cp3.n_beads = 1
    cp3.kT_fluid = 0.0
    rc = L.lbmd_lb_step_noalloc(C.byref(cp3), C.c_void_p(f.data_ptr()), C.c_void_p(g.data_ptr()), None)
    assert rc == lb.lbmd.LBMD_EUNSUPPORTED
    # a box within the scratch whose y extent exceeds the launch grid
    cp4, keep4 = lb.make_params(dict(nx=8, ny=600000, nz=1, wall_x=-1))
    rc = L.lbmd_lb_step_noalloc(C.byref(cp4), C.c_void_p(f.data_ptr()), C.c_void_p(g.data_ptr()), None)
    assert rc == lb.lbmd.LBMD_EINVAL
    del keep, keep2, keep3, keep4
