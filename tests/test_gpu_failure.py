"""Failure states of the coupled step on the GPU, reached from the host side
(parameters and initial state only; nothing here faults, traps or hangs a
GPU):

* SHAKE failure (Sec. II, SHAKE / RATTLE): one constraint iteration against
  a tolerance of 1e-12, with bead velocities that stretch every bond by a
  third of its length in one substep.  The oracle's Gauss-Seidel sweep and the
  GPU's Newton step both stop above their acceptance bounds, and both state
  machines report LBMD_SHAKE_FAIL after the first step.
* Non-finite beads: an initial velocity of 1e25 lattice units per step; the
  squared bond lengths of the next substep exceed the FP32 range, the
  constraint solve returns NaN and the state is LBMD_NAN after one step.
* Non-finite populations: tau = 0.5001 (omega ~ 2) with a strong random
  initial flow is linearly unstable (the FP64 oracle overflows after ~400
  steps on the same box).  The stream-collide flags a node whose pulled
  populations (hence density) are not finite, so the state turns LBMD_NAN
  one step after the populations first read non-finite (or in the same step,
  when the FP32 density sum overflows first).
* In an ensemble the failing realisations stop at their failure step while
  the others run on, bit-identical to their single-box runs.
"""
import numpy as np
import pytest

import oracle
import seeded_inputs as si

pytestmark = pytest.mark.gpu

PAPER_EPS = 2e-3


def _lb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0710_1272_gb300 as lb
    return lb


def shake_case(seed=7):
    """Small translocation box; bead velocities +-2 along x, alternating, so
    that every bond changes by 0.8 (its length is 1.2) in one substep."""
    p = si.small_translocation(seed)
    p.update(lj_eps=PAPER_EPS, shake_max_iter=1, shake_tol=1e-12)
    pos = si.saw_chain(p, seed)
    vel = np.zeros_like(pos)
    vel[:, 0] = np.where(np.arange(p["n_beads"]) % 2 == 0, 2.0, -2.0)
    return p, pos, vel


def unstable_flow(shape, seed=5):
    return si.random_flow(shape, seed=seed, u_max=0.3)


def test_shake_failure_matches_oracle_state_machine():
    lb = _lb()
    p, pos, vel = shake_case()
    orc = oracle.OracleSim(p, init_pos=pos, init_vel=vel)
    orc.step(1)
    assert orc.status()["state"] == oracle.SHAKE_FAIL  # the oracle's verdict
    sim = lb.Simulation(p, init_pos=pos, init_vel=vel)
    sim.step(1)
    st = sim.status()
    assert st["state"] == lb.SHAKE_FAIL and st["step"] == 1
    assert sim.solver_stats()["failed_steps"] == 1
    r, v = sim.beads()
    assert np.all(np.isfinite(r)) and np.all(np.isfinite(v))
    # the state word stays; the context keeps stepping without a CUDA error
    sim.step(5)
    st = sim.status()
    assert st["state"] == lb.SHAKE_FAIL and st["step"] == 6


def test_huge_bead_velocity_gives_nan_state():
    lb = _lb()
    p = si.small_translocation(2)
    pos = si.saw_chain(p, 2)
    vel = np.zeros_like(pos)
    vel[3] = (1e25, -1e25, 1e25)
    sim = lb.Simulation(p, init_pos=pos, init_vel=vel)
    sim.step(1)
    assert sim.status()["state"] == lb.NAN
    r, v = sim.beads()
    assert not (np.all(np.isfinite(r)) and np.all(np.isfinite(v)))
    sim.step(3)
    assert sim.status()["state"] == lb.NAN and sim.status()["step"] == 4


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_nonfinite_populations_detected_one_step_later(storage):
    lb = _lb()
    p = dict(nx=16, ny=8, nz=8, wall_x=-1, n_beads=0, tau=0.5001, storage=storage)
    rho, u = unstable_flow((8, 8, 16))
    sim = lb.Simulation(p, init_rho=rho, init_u=u)
    first_bad_f = first_nan_state = None
    for n in range(1, 801):
        sim.step(1)
        st = sim.status()["state"]
        if first_nan_state is None and st == lb.NAN:
            first_nan_state = n
        if first_bad_f is None and not np.all(np.isfinite(sim.populations())):
            first_bad_f = n
        if first_nan_state is not None and first_bad_f is not None:
            break
    assert first_bad_f is not None, "the unstable flow stayed finite"
    # a non-finite population makes the next step's density non-finite; the
    # FP32 density sum can also overflow one step before an element does
    assert first_bad_f <= first_nan_state <= first_bad_f + 1
    sim.step(10)
    assert sim.status()["state"] == lb.NAN


def test_nonfinite_populations_stop_a_coupled_box():
    """gamma = 0: the exploding flow drags no bead apart (with drag the
    constraint solve fails first and the state is LBMD_SHAKE_FAIL); once the
    populations are not finite the state is LBMD_NAN -- the beads may be
    non-finite too, since u_i enters the drag force (0 * NaN is NaN)."""
    lb = _lb()
    p = si.small_translocation(1)
    p.update(tau=0.5001, lj_eps=PAPER_EPS, gamma=0.0)
    pos = si.saw_chain(p, 1)
    rho, u = unstable_flow((16, 16, 32), seed=9)
    sim = lb.Simulation(p, init_pos=pos, init_rho=rho, init_u=u)
    for _ in range(16):
        sim.step(50)
        if sim.status()["state"] != lb.RUNNING:
            break
    assert sim.status()["state"] == lb.NAN
    assert not np.all(np.isfinite(sim.populations()))


def test_ensemble_failing_members_stop_others_run_on():
    lb = _lb()
    p_shake, pos_shake, vel_shake = shake_case()
    p_nan = si.small_translocation(2)
    pos_nan = si.saw_chain(p_nan, 2)
    vel_nan = np.zeros_like(pos_nan)
    vel_nan[3] = (1e25, -1e25, 1e25)
    p_ok = dict(si.small_translocation(4), lj_eps=PAPER_EPS)
    pos_ok = si.saw_chain(p_ok, 4)
    p_flow = dict(si.small_translocation(1), tau=0.5001, lj_eps=PAPER_EPS, gamma=0.0)
    pos_flow = si.saw_chain(p_flow, 1)
    rho, u = unstable_flow((16, 16, 32), seed=9)
    members = [p_shake, p_nan, p_ok, p_flow]
    starts = [pos_shake, pos_nan, pos_ok, pos_flow]
    ens = lb.Ensemble(members, starts, init_vel=[vel_shake, vel_nan, None, None],
                      init_rho=[None, None, None, rho], init_u=[None, None, None, u])
    ens.run(800, check_every=16)
    res = ens.results()
    assert res["state"][0] == lb.SHAKE_FAIL and res["steps"][0] == 1
    assert res["state"][1] == lb.NAN and res["steps"][1] == 1
    assert res["state"][3] == lb.NAN and res["steps"][3] < 800
    assert np.all(np.isfinite(ens.beads(3)[0]))  # the populations, not the chain
    # the healthy realisation ran on to its end (translocation or the cap)
    assert res["steps"][2] == (res["t_transloc"][2] if res["state"][2] == lb.TRANSLOCATED else 800)
    # each realisation equals its single-box run, failures included
    for k, (p, pos) in enumerate(zip(members, starts)):
        kw = {}
        if k == 0:
            kw = dict(init_vel=vel_shake)
        elif k == 1:
            kw = dict(init_vel=vel_nan)
        elif k == 3:
            kw = dict(init_rho=rho, init_u=u)
        sim = lb.Simulation(p, init_pos=pos, **kw)
        sim.step(int(res["steps"][k]))
        st = sim.status()
        assert st["state"] == res["state"][k], k
        np.testing.assert_array_equal(ens.beads(k)[0], sim.beads()[0])
        if k == 2:
            np.testing.assert_array_equal(ens.populations(k), sim.populations())
