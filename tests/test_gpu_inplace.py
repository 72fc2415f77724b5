"""In-place (AA-pattern) streaming on the GPU: the one-buffer path against the
FP64 oracle on the same seeded inputs, and against the two-buffer pull path.

The in-place path performs the same arithmetic on the same values as the pull
path -- only the slots the values are kept in differ -- so the two agree bit
for bit in every storage type, at every step parity, through graph replays of
any length, with the thermal source, and with a coupled chain (the spread sums
each node's impulses in fixed point and adds them once, independent of the
order of its atomics).  Against the oracle the bars are those of the pull path:
populations within 1e-5 relative after one step and 1e-4 after 1000, beads
within 1e-4 over 100 steps.
"""
import numpy as np
import pytest

import oracle
import seeded_inputs as si

pytestmark = pytest.mark.gpu

GPU_ONLY = ("storage", "init_tg_amp", "diag_every", "diag_capacity", "streaming")


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0710_1272_gb300 as lb
    return lb


def rel_err(fg, fo):
    m = fo != 0
    assert np.all(fg[~m] == 0)
    return float(np.max(np.abs(fg[m].astype(np.float64) - fo[m]) / np.abs(fo[m])))


def aa_and_oracle(p, init_pos=None, init_rho=None, init_u=None, **gpu_kw):
    lb = _gpu()
    gp = dict(p, streaming="aa", **gpu_kw)
    sim = lb.Simulation(gp, init_pos=init_pos, init_rho=init_rho, init_u=init_u)
    op = {k: v for k, v in p.items() if k not in GPU_ONLY}
    orc = oracle.OracleSim(op, init_pos=init_pos, init_rho=init_rho, init_u=init_u)
    return sim, orc


def aa_and_pull(p, init_pos=None, init_rho=None, init_u=None, **gpu_kw):
    lb = _gpu()
    a = lb.Simulation(dict(p, streaming="aa", **gpu_kw), init_pos=init_pos, init_rho=init_rho,
                      init_u=init_u)
    b = lb.Simulation(dict(p, streaming="pull", **gpu_kw), init_pos=init_pos, init_rho=init_rho,
                      init_u=init_u)
    return a, b


LB_CASES = [
    dict(nx=4, ny=4, nz=4, wall_x=-1, tau=0.8, body_force=(1e-4, 0, 0)),
    dict(nx=5, ny=4, nz=3, wall_x=2, pore_d=1, pore_y0=1, pore_z0=1, tau=0.6),
    dict(nx=33, ny=17, nz=5, wall_x=20, pore_d=3, y_walls=1, tau=1.0, forcing="guo",
         body_force=(1e-5, 2e-6, 0)),
    dict(nx=32, ny=16, nz=16, wall_x=16, pore_d=3, tau=1.0, body_force=(1e-6, 0, 0)),
    dict(nx=70, ny=9, nz=4, wall_x=0, wall_thickness=2, pore_d=2, tau=0.7),
    dict(nx=1, ny=3, nz=2, wall_x=-1, tau=0.9, body_force=(0, 1e-4, 0)),
]


@pytest.mark.parametrize("case", range(len(LB_CASES)))
def test_inplace_steps_match_oracle(case):
    """Both step kinds (even: local, odd: pull + push with bounce-back) and
    the read-outs of both layouts, on boxes with walls, a pore, y-walls,
    ragged widths, Guo forcing and a one-node-wide periodic box."""
    p = LB_CASES[case]
    shape = (p["nz"], p["ny"], p["nx"])
    rho, u = si.random_flow(shape, seed=30 + case, u_max=0.04)
    sim, orc = aa_and_oracle(p, init_rho=rho, init_u=u)
    assert rel_err(sim.populations(), orc.populations()) < 2e-6
    for n in range(1, 5):
        sim.step(1)
        orc.step(1)
        assert rel_err(sim.populations(), orc.populations()) < 1e-5 * n, n
        rg, ug = sim.fields()
        ro, uo = orc.fields()
        np.testing.assert_allclose(rg, ro, atol=2e-6 * n)
        np.testing.assert_allclose(ug, uo, atol=2e-6 * n)


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("case", range(len(LB_CASES)))
def test_inplace_equals_pull_bitwise(case, storage):
    p = LB_CASES[case]
    shape = (p["nz"], p["ny"], p["nx"])
    rho, u = si.random_flow(shape, seed=40 + case, u_max=0.04)
    a, b = aa_and_pull(p, init_rho=rho, init_u=u, storage=storage)
    for n in (1, 1, 2, 3, 17, 1, 33):  # graph replays of 1, 2 and 16 steps, both parities
        a.step(n)
        b.step(n)
        assert np.array_equal(a.populations(), b.populations()), n
        ra, ua = a.fields()
        rb, ub = b.fields()
        assert np.array_equal(ra, rb) and np.array_equal(ua, ub)


def test_inplace_1000_steps_match_oracle():
    p = LB_CASES[3]
    rho, u = si.random_flow((p["nz"], p["ny"], p["nx"]), seed=7, u_max=0.03)
    sim, orc = aa_and_oracle(p, init_rho=rho, init_u=u)
    sim.step(1000)
    orc.step(1000)
    assert rel_err(sim.populations(), orc.populations()) < 1e-4


def test_inplace_initial_fields_in_several_slabs():
    """Given initial fields go through the staging buffer one z-slab at a
    time (here 128 planes, then a ragged 33): the result equals the pull
    path's initial state and its first steps."""
    p = dict(nx=128, ny=64, nz=161, wall_x=64, pore_d=5, tau=0.9)
    rho, u = si.random_flow((p["nz"], p["ny"], p["nx"]), seed=3, u_max=0.03)
    a, b = aa_and_pull(p, init_rho=rho, init_u=u)
    assert np.array_equal(a.populations(), b.populations())
    a.step(3)
    b.step(3)
    assert np.array_equal(a.populations(), b.populations())


def test_inplace_thermal_source_equals_pull():
    """The thermal source draws its normals from (node, step) counters, so
    the in-place path reproduces the pull path's fluctuating run exactly."""
    p = dict(nx=32, ny=16, nz=16, wall_x=16, pore_d=3, tau=0.8, kT_fluid=1e-5, seed=11)
    for storage in ("f32", "f16"):
        a, b = aa_and_pull(p, storage=storage)
        for n in (1, 2, 5):
            a.step(n)
            b.step(n)
            assert np.array_equal(a.populations(), b.populations()), (storage, n)


# -- coupled LB + MD ------------------------------------------------------------

PAPER_EPS = 2e-3


def small_case(seed=0, **kw):
    p = si.small_translocation(seed)
    p.update(kw)
    return p, si.saw_chain(p, seed)


def test_inplace_coupled_one_and_two_steps():
    """Gather from both layouts and spread into both (after an even step the
    source goes to the swapped slot, after an odd step to the neighbour the
    population is pushed to, or back into the node next to a solid)."""
    p, pos = small_case(0)
    sim, orc = aa_and_oracle(p, init_pos=pos)
    for n in (1, 2, 3):
        sim.step(1)
        orc.step(1)
        assert rel_err(sim.populations(), orc.populations()) < 1e-5, n
        rg, vg = sim.beads()
        ro, vo = orc.beads()
        np.testing.assert_allclose(rg, ro, atol=1e-5)
        np.testing.assert_allclose(vg, vo, atol=1e-5)
        ug, Jg = sim.bead_aux()
        uo, Jo = orc.bead_aux()
        np.testing.assert_allclose(ug, uo, atol=1e-7)
        np.testing.assert_allclose(Jg, Jo, atol=1e-6)


@pytest.mark.parametrize("seed", [0, 1])
def test_inplace_coupled_trajectory_100_steps(seed):
    p, pos = small_case(seed, lj_eps=PAPER_EPS)
    sim, orc = aa_and_oracle(p, init_pos=pos)
    for _ in range(10):
        sim.step(10)
        orc.step(10)
        assert np.abs(sim.beads()[0] - orc.beads()[0]).max() < 1e-4
    assert sim.status()["state"] == orc.status()["state"]


def test_inplace_coupled_populations_1000_steps():
    p, pos = small_case(0, lj_eps=PAPER_EPS, f_drive=0.0)
    sim, orc = aa_and_oracle(p, init_pos=pos)
    sim.step(1000)
    orc.step(1000)
    assert rel_err(sim.populations(), orc.populations()) < 1e-4


@pytest.mark.parametrize("variant", [dict(coupling="ngp"), dict(forcing="guo", body_force=(2e-6, 0, 0)),
                                     dict(kappa_phi=5e-4), dict(storage="f16")])
def test_inplace_coupled_equals_pull(variant):
    p, pos = small_case(2, lj_eps=PAPER_EPS)
    p.update({k: v for k, v in variant.items() if k != "storage"})
    kw = {"storage": variant["storage"]} if "storage" in variant else {}
    a, b = aa_and_pull(p, init_pos=pos, **kw)
    for n in (1, 1, 16, 3):
        a.step(n)
        b.step(n)
        assert np.array_equal(a.populations(), b.populations()), n
        assert np.array_equal(a.beads()[0], b.beads()[0]), n
        assert np.array_equal(a.beads()[1], b.beads()[1]), n
    assert a.status() == b.status()


def test_inplace_paper_sized_box():
    """256 x 128 x 128 box, 5x5 pore, 400 beads, in the benchmark's launch
    configuration (graph replay): the full field and every bead after three
    steps against the oracle."""
    p = si.paper_translocation(0)
    pos = si.saw_chain(p, 0)
    sim, orc = aa_and_oracle(p, init_pos=pos)
    sim.step(3)
    orc.step(3)
    assert rel_err(sim.populations(), orc.populations()) < 1e-5
    assert np.abs(sim.beads()[0] - orc.beads()[0]).max() < 1e-5


def test_inplace_solvent_free_and_diagnostics():
    p, pos = small_case(1, lj_eps=PAPER_EPS)
    a, b = aa_and_pull(dict(p, hydrodynamics=0, diag_every=5, diag_capacity=8), init_pos=pos)
    a.step(20)
    b.step(20)
    np.testing.assert_array_equal(a.beads()[0], b.beads()[0])
    da, db = a.diagnostics(), b.diagnostics()
    assert set(da) == set(db) and len(da["step"]) == 4
    for k in da:
        np.testing.assert_array_equal(da[k], db[k])
