"""Pins of the oracle's Sec. III chain diagnostics: the radii of gyration of
the untranslocated and translocated parts (R_U, R_T), the effective radius
R_E = (R_T^(1/mu) + R_U^(1/mu))^mu with mu = 0.6, the fluid's work rate
S_H (Eq. 13), the drive's work rate S_E (Eq. 14) and the kinetic energy K.
Checked on configurations whose values are known in closed form."""
import math

import numpy as np
import pytest

import oracle
import seeded_inputs as si


def sim(n, **kw):
    p = si.small_translocation(0, n_beads=n)
    p.update(kw)
    pos = np.tile([[20.0, 7.0, 7.0]], (n, 1)) + np.arange(n)[:, None] * [0.0, 1.0, 0.0]
    return oracle.OracleSim(p, init_pos=pos), p


def line(n, b, start, axis):
    pos = np.tile(np.asarray(start, float), (n, 1))
    pos[:, axis] += b * np.arange(n)
    return pos


def test_radius_of_gyration_of_straight_segments():
    # n equally spaced points: R^2 = b^2 (n^2 - 1) / 12
    n, k, b = 9, 4, 1.2
    s, p = sim(n)
    pos = np.vstack([line(k, b, [12.0, 3.0, 2.0], 2),        # translocated, x < 16
                     line(n - k, b, [21.0, 2.0, 5.0], 1)])   # untranslocated
    z = np.zeros_like(pos)
    d = s.diagnostics(pos, z, z)
    assert d["n_trans"] == k
    assert d["r_t"] == pytest.approx(b * math.sqrt((k * k - 1) / 12), rel=1e-14)
    assert d["r_u"] == pytest.approx(b * math.sqrt(((n - k) ** 2 - 1) / 12), rel=1e-14)


def test_effective_radius_special_cases():
    s, p = sim(8)
    # all beads untranslocated: R_T = 0 and R_E = R_U
    pos = line(8, 1.5, [20.0, 2.0, 2.0], 1)
    z = np.zeros_like(pos)
    d = s.diagnostics(pos, z, z)
    assert d["r_t"] == 0.0 and d["r_e"] == pytest.approx(d["r_u"], rel=1e-15)
    # two equal halves: R_E = 2^mu R with mu = 0.6
    pos = np.vstack([line(4, 1.5, [10.0, 2.0, 2.0], 1), line(4, 1.5, [20.0, 2.0, 2.0], 2)])
    d = s.diagnostics(pos, z, z)
    assert d["r_t"] == pytest.approx(d["r_u"], rel=1e-14)
    assert d["r_e"] == pytest.approx(2 ** 0.6 * d["r_u"], rel=1e-14)


def test_radius_is_translation_invariant_and_order_free():
    s, p = sim(10)
    rng = np.random.default_rng(3)
    pos = np.column_stack([rng.uniform(18, 30, 10), rng.uniform(0, 16, 10), rng.uniform(0, 16, 10)])
    z = np.zeros_like(pos)
    d0 = s.diagnostics(pos, z, z)
    d1 = s.diagnostics(pos + [0.7, -3.1, 40.0], z, z)
    d2 = s.diagnostics(pos[::-1].copy(), z, z)
    for key in ("r_u", "r_t", "r_e"):
        assert d1[key] == pytest.approx(d0[key], rel=1e-12, abs=1e-12)
        assert d2[key] == pytest.approx(d0[key], rel=1e-12, abs=1e-12)


def test_work_rates_and_kinetic_energy():
    n = 6
    s, p = sim(n, bead_mass=2.0, gamma=0.1)
    pos = line(n, 1.2, [22.0, 3.0, 3.0], 1)          # outside the drive channel
    ones = np.tile([1.0, 0.0, 0.0], (n, 1))
    d = s.diagnostics(pos, ones, ones)
    assert d["s_h"] == pytest.approx(2.0 * 0.1 * n, rel=1e-15)   # m gamma sum v.u
    assert d["s_e"] == 0.0
    assert d["kinetic"] == pytest.approx(0.5 * 2.0 * n, rel=1e-15)
    perp = np.tile([0.0, 1.0, 0.0], (n, 1))
    assert s.diagnostics(pos, ones, perp)["s_h"] == 0.0
    v = np.zeros((n, 3))
    v[0] = [3.0, 4.0, 0.0]
    assert s.diagnostics(pos, v, np.zeros((n, 3)))["kinetic"] == pytest.approx(25.0, rel=1e-15)


def test_drive_work_rate_inside_the_channel():
    s, p = sim(2)
    y0, z0, d = si.pore_geometry(p)
    c = [p["wall_x"], y0 + (d - 1) / 2, z0 + (d - 1) / 2]
    pos = np.array([c, [25.0, 3.0, 3.0]])
    v = np.array([[-0.3, 0.2, 0.1], [-0.3, 0.0, 0.0]])
    out = s.diagnostics(pos, v, np.zeros((2, 3)))
    # F_drive = -f_drive x on bead 0 only; moving along -x: positive work
    assert out["s_e"] == pytest.approx(p["f_drive"] * 0.3, rel=1e-15)


def test_state_diagnostics_match_the_state():
    p = si.small_translocation(2)
    pos = si.saw_chain(p, 2)
    s = oracle.OracleSim(p, init_pos=pos)
    s.step(30)
    r, v = s.beads()
    ui, _ = s.bead_aux()
    d = s.diagnostics()
    e = s.diagnostics(r, v, ui)
    assert d == e
    assert d["n_trans"] == s.status()["n_trans"]
    assert d["s_h"] != 0.0 and d["kinetic"] > 0.0
