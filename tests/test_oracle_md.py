"""Pins of the oracle's polymer MD (Sec. II, Eqs. 1-4; SHAKE/RATTLE; Sec. III
drive and bookkeeping): published Philox vectors, Gaussian moments, closed-form
potential values, forces = -grad(energy) by finite differences, SHAKE against
an independent Newton solve, the exact stationary temperature of the discrete
Langevin substep, and the translocation state machine."""
import math
import os

import numpy as np
import pytest

import oracle
import seeded_inputs as si

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
NO_BONDS = (np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0))


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert out.tolist() == v[6:10]


def test_gaussian_moments():
    """Box-Muller deviates: mean 0, variance 1, components uncorrelated,
    within 5 sigma of sampling error."""
    n = 40000
    xi = np.array([oracle.gauss3(1234, i % 400, i // 400, 3) for i in range(n)])
    m = xi.mean(0)
    assert np.all(np.abs(m) < 5 / math.sqrt(n))
    var = xi.var(0)
    assert np.all(np.abs(var - 1) < 5 * math.sqrt(2 / n))
    cxy = (xi[:, 0] * xi[:, 1]).mean()
    assert abs(cxy) < 5 / math.sqrt(n)
    # fourth moment of a normal is 3
    assert np.all(np.abs((xi ** 4).mean(0) - 3) < 5 * math.sqrt(96 / n))
    # distinct counters give distinct draws; same counter repeats
    assert np.all(oracle.gauss3(1, 2, 3, 4) == oracle.gauss3(1, 2, 3, 4))
    assert not np.allclose(oracle.gauss3(1, 2, 3, 4), oracle.gauss3(1, 2, 3, 4, stream=1))


def _pair_sim(eps=1.0, sigma=1.8):
    p = dict(nx=40, ny=40, nz=40, wall_x=-1, n_beads=2, lj_eps=eps, lj_sigma=sigma,
             f_drive=0.0)
    return oracle.OracleSim(p, init_pos=np.array([[10.0, 10, 10], [12.0, 10, 10]]), bonds=NO_BONDS)


def test_wca_closed_form_values():
    """Eq. 2 truncated at r_c = 2^(1/6) sigma and shifted by eps: V(sigma) = eps,
    V -> 0 and F -> 0 at r_c, nothing beyond; the force is repulsive."""
    s = _pair_sim()
    sig = 1.8
    rc = 2 ** (1 / 6) * sig
    E, F = s.forces(np.array([[10.0, 10, 10], [10 + sig, 10, 10]]))
    assert abs(E - 1.0) < 1e-14
    # at sigma: F = 24 eps / sigma (2 - 1) = 24 / sigma, repulsive
    np.testing.assert_allclose(F[0], [-24 / sig, 0, 0], rtol=1e-14)
    np.testing.assert_allclose(F[1], [24 / sig, 0, 0], rtol=1e-14)
    E, F = s.forces(np.array([[10.0, 10, 10], [10 + rc * (1 - 1e-9), 10, 10]]))
    assert abs(E) < 1e-7 and np.abs(F).max() < 1e-6
    E, F = s.forces(np.array([[10.0, 10, 10], [10 + rc * (1 + 1e-9), 10, 10]]))
    assert E == 0 and np.all(F == 0)
    # minimum image across the periodic boundary
    E, F = s.forces(np.array([[0.5, 10, 10], [39.5 - 0.3, 10, 10]]))
    assert F[0][0] > 0 and abs(F[0][0] + F[1][0]) < 1e-14


def _numgrad(s, pos, h=1e-6):
    g = np.zeros_like(pos)
    for i in range(pos.shape[0]):
        for a in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, a] += h
            pm[i, a] -= h
            g[i, a] = (s.forces(pp)[0] - s.forces(pm)[0]) / (2 * h)
    return g


def test_forces_are_minus_energy_gradient():
    """Bead-bead WCA (non-bonded pairs), bending (Eq. 3) and bead-wall WCA are
    conservative: F = -dE/dr, checked by central differences."""
    p = dict(si.small_translocation(0, n_beads=8))
    p.update(kappa_phi=0.7, f_drive=0.0, lj_eps=0.01)
    rng = np.random.default_rng(3)
    pos = si.saw_chain(p, 2)
    pos += rng.normal(0, 0.15, pos.shape)
    pos[0] = [16.9, 7.4, 6.8]  # in the pore mouth: feels the wall and the pore lining
    pos[3] = pos[5] + [1.5, 0.3, -0.2]  # a non-bonded overlap
    s = oracle.OracleSim(p, init_pos=pos)
    E, F = s.forces(pos)
    assert E > 0
    np.testing.assert_allclose(F, -_numgrad(s, pos), rtol=1e-6, atol=1e-8)
    # forces between beads (and bending) sum to zero without the wall
    q = dict(p, wall_x=-1)
    s2 = oracle.OracleSim(q, init_pos=pos)
    assert np.abs(s2.forces(pos)[1].sum(0)).max() < 1e-12


def test_bending_angle_definition():
    """Eq. 3: phi is the angle between consecutive bonds (0 for a straight
    chain); a right-angle bend stores kappa (pi/2)^2 / 2."""
    p = dict(nx=30, ny=30, nz=30, wall_x=-1, n_beads=3, kappa_phi=2.0, lj_eps=0.0)
    straight = np.array([[5.0, 5, 5], [6.2, 5, 5], [7.4, 5, 5]])
    bent = np.array([[5.0, 5, 5], [6.2, 5, 5], [6.2, 6.2, 5]])
    s = oracle.OracleSim(p, init_pos=straight)
    E, F = s.forces(straight)
    assert abs(E) < 1e-20 and np.abs(F).max() < 1e-12
    E, F = s.forces(bent)
    assert abs(E - 2.0 * (math.pi / 2) ** 2 / 2) < 1e-13


def test_drive_region():
    """Sec. III pulling force: -f_drive along x inside the 3-node channel
    through the pore, zero elsewhere."""
    p = dict(si.small_translocation(0, n_beads=1))
    p.update(lj_eps=0.0, f_drive=0.02)
    s = oracle.OracleSim(p, init_pos=np.array([[17.0, 7.0, 7.0]]), bonds=NO_BONDS)
    y0, z0, d = si.pore_geometry(p)
    inside = [[16.0, 7, 7], [14.6, 7, 7], [17.4, 7.2, 6.6], [16.0, y0 - 0.49, z0 + d - 0.51]]
    outside = [[18.6, 7, 7], [13.4, 7, 7], [16.0, y0 - 0.51, 7], [16.0, 7, z0 + d - 0.49], [3.0, 7, 7]]
    for r in inside:
        np.testing.assert_allclose(s.forces(np.array([r]))[1][0], [-0.02, 0, 0], atol=1e-17)
    for r in outside:
        assert np.all(s.forces(np.array([r]))[1][0] == 0)


def _newton_constraints(r_old, r_tilde, b0, m=1.0):
    """Independent solve of the SHAKE equations |d_b(lambda)|^2 = b0^2, with
    d_b moving along the old bond vectors, by Newton on the multipliers
    (dense linear algebra)."""
    N = r_old.shape[0]
    s = r_old[1:] - r_old[:-1]
    lam = np.zeros(N - 1)

    def positions(lam):
        r = r_tilde.copy()
        r[:-1] += (lam[:, None] * s) / m
        r[1:] -= (lam[:, None] * s) / m
        return r

    for _ in range(50):
        r = positions(lam)
        d = r[1:] - r[:-1]
        G = (d * d).sum(1) - b0 ** 2
        if np.abs(G).max() < 1e-15:
            break
        Jm = np.zeros((N - 1, N - 1))
        for b in range(N - 1):
            Jm[b, b] = -2 * d[b] @ s[b] * (2 / m)
            if b > 0:
                Jm[b, b - 1] = 2 * d[b] @ s[b - 1] / m
            if b < N - 2:
                Jm[b, b + 1] = 2 * d[b] @ s[b + 1] / m
        lam -= np.linalg.solve(Jm, G)
    return positions(lam)


def test_shake_matches_newton_solution():
    """P8: Gauss-Seidel SHAKE converges to the unique nearby solution of the
    constraint equations, the same one a Newton solve finds."""
    p = dict(si.small_translocation(0, n_beads=40))
    p.update(nx=64, ny=64, nz=64, wall_x=-1, shake_tol=1e-13)
    r_old = si.saw_chain(dict(p, wall_x=-1), 6)
    rng = np.random.default_rng(4)
    r_new = r_old + 0.05 * rng.standard_normal(r_old.shape)
    s = oracle.OracleSim(p, init_pos=r_old)
    rc, r_shake, sweeps = s.shake(r_old, r_new)
    assert rc == 0 and sweeps > 1
    d = np.linalg.norm(np.diff(r_shake, axis=0), axis=1)
    assert np.abs(d - 1.2).max() < 1e-12
    r_ref = _newton_constraints(r_old, r_new, 1.2)
    np.testing.assert_allclose(r_shake, r_ref, atol=1e-12)
    # momentum-conserving corrections
    np.testing.assert_allclose(r_shake.sum(0), r_new.sum(0), atol=1e-11)


def test_rattle_removes_bond_velocities():
    p = dict(nx=64, ny=64, nz=64, wall_x=-1, n_beads=25, shake_tol=1e-15)
    r = si.saw_chain(dict(si.small_translocation(0, n_beads=25), nx=64, ny=64, nz=64, wall_x=-1), 7)
    v = np.random.default_rng(5).standard_normal(r.shape) * 0.1
    s = oracle.OracleSim(p, init_pos=r)
    rc, v2, sweeps = s.rattle(r, v)
    assert rc == 0
    d = np.diff(r, axis=0)
    assert np.abs((d * np.diff(v2, axis=0)).sum(1)).max() < 1e-14
    np.testing.assert_allclose(v2.sum(0), v.sum(0), atol=1e-13)
    # the projection is orthogonal: applying it twice changes nothing
    rc, v3, _ = s.rattle(r, v2)
    np.testing.assert_allclose(v3, v2, atol=1e-14)


def test_constraints_hold_along_a_run():
    """P8: after every LB step bond lengths equal b to 1e-10 and relative
    velocities are perpendicular to the bonds."""
    p = si.small_translocation(1)
    pos = si.saw_chain(p, 1)
    s = oracle.OracleSim(p, init_pos=pos)
    for _ in range(20):
        assert s.step(5) == 0
        r, v = s.beads()
        d = np.diff(r, axis=0)
        assert np.abs(np.linalg.norm(d, axis=1) - 1.2).max() < 1e-10
        assert np.abs((d * np.diff(v, axis=0)).sum(1)).max() < 1e-10
    assert s.status()["state"] == oracle.RUNNING


def test_discrete_langevin_temperature_exact():
    """The Euler-Langevin substep v' = (1 - gamma dt) v + sqrt(2 gamma kT dt) xi
    (m = 1, u = 0, no other force) has the exact stationary variance
    kT / (1 - gamma dt / 2); this pins the noise amplitude of the
    fluctuation-dissipation reading and the drag term (Eq. 4)."""
    N, kT, gamma = 200, 1.0, 1.0
    p = dict(nx=40, ny=40, nz=40, wall_x=-1, n_beads=N, lj_eps=0.0, lj_sigma=1e-3,
             gamma=gamma, kT=kT, hydrodynamics=0, seed=99)
    pos = np.random.default_rng(0).uniform(0, 40, (N, 3))
    vel = np.random.default_rng(1).normal(0, math.sqrt(kT), (N, 3))
    s = oracle.OracleSim(p, init_pos=pos, init_vel=vel, bonds=NO_BONDS)
    s.step(20)
    acc = []
    for _ in range(300):
        s.step(2)
        acc.append((s.beads()[1] ** 2).mean())
    dt = 1 / 5
    expected = kT / (1 - gamma * dt / 2)
    # samples 10 substeps apart, correlation (1 - 0.2)^20 ~ 0.01
    err = 5 * expected * math.sqrt(2 / (3 * N * len(acc)))
    assert abs(np.mean(acc) - expected) < err
    assert abs(np.mean(acc) - kT) > 5 * err  # the discretisation bias is resolved


def _free_beads(xs, vxs):
    p = dict(si.small_translocation(0, n_beads=len(xs)))
    p.update(lj_eps=0.0, f_drive=0.0, gamma=0.0, kT=0.0, hydrodynamics=0)
    return oracle.OracleSim(p, init_pos=np.array([[x, 7.0, 7.0] for x in xs]),
                            init_vel=np.array([[v, 0, 0] for v in vxs]), bonds=NO_BONDS)


def test_translocation_completion():
    s = _free_beads([15.0], [0.0])
    s.step(1)
    st = s.status()
    assert st == dict(step=1, n_trans=1, state=oracle.TRANSLOCATED, t_transloc=1)
    s.step(3)
    assert s.status()["t_transloc"] == 1


def test_retraction():
    """After one bead crossed, every bead back beyond the drive channel
    (x > x_wall + 1.5) ends the event as a retraction."""
    s = _free_beads([15.7, 25.0], [0.25, 0.0])  # bead 0 crosses back: x(n) = 15.7 + 0.25 n
    states = []
    for n in range(1, 10):
        s.step(1)
        states.append((s.status()["n_trans"], s.status()["state"]))
    assert states[0] == (1, oracle.RUNNING)
    assert states[1] == (0, oracle.RUNNING)
    first = [i + 1 for i, (nt, st) in enumerate(states) if st == oracle.RETRACTED][0]
    assert first == 8  # 15.7 + 0.25 * 8 = 17.7 > 17.5 > 15.7 + 0.25 * 7


def test_nan_status():
    p = si.small_translocation(0, n_beads=4)
    pos = si.saw_chain(p, 0)
    pos[2, 1] = np.nan
    s = oracle.OracleSim(p, init_pos=pos)
    s.step(1)
    assert s.status()["state"] == oracle.NAN


def test_saw_inputs_are_valid():
    p = si.small_translocation(0)
    for seed in range(3):
        pos = si.saw_chain(p, seed)
        d = np.linalg.norm(np.diff(pos, axis=0), axis=1)
        assert np.abs(d - 1.2).max() < 1e-12
        assert np.all(pos[2:, 0] > 16 + 2.0)
        rc = 2 ** (1 / 6) * 1.8
        for i in range(len(pos)):
            for j in range(i + 2, len(pos)):
                assert np.linalg.norm(pos[i] - pos[j]) >= rc
