"""The library's own chain start (lbmd_params.init_pos == NULL; Sec. III: the
chain starts on the cis side with one end in the pore).

Through the C ABI: a context created without init_pos holds a start that is
a self-avoiding walk as specified -- bond lengths b, no non-bonded pair
within 2^(1/6) sigma (minimum image), beads 2.. at least that far from the
wall plane and from every solid node, bead 0 at the pore mouth, zero
velocities -- that depends on the seed only, and that steps exactly as the
oracle does when the oracle starts from the positions read back."""
import numpy as np
import pytest

import oracle
import seeded_inputs as si

pytestmark = pytest.mark.gpu

RC_FACTOR = 2 ** (1 / 6)


def _lb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_0710_1272_gb300 as lb
    return lb


def rel_err(fg, fo):
    m = fo != 0
    assert np.all(fg[~m] == 0)
    return float(np.max(np.abs(fg[m].astype(np.float64) - fo[m]) / np.abs(fo[m])))


def check_walk(p, r):
    N = p["n_beads"]
    L = np.array([p["nx"], p["ny"], p["nz"]], dtype=np.float64)
    rc = RC_FACTOR * p["lj_sigma"]
    b = p["bond_len"]
    t = p.get("wall_thickness", 1)
    xw = p["wall_x"]
    y0, z0, d = si.pore_geometry(p)
    assert r.shape == (N, 3)
    np.testing.assert_allclose(r[0], (xw + t, y0 + (d - 1) / 2, z0 + (d - 1) / 2), atol=1e-12)
    np.testing.assert_allclose(r[1], r[0] + (b, 0, 0), atol=1e-12)
    bonds = np.linalg.norm(np.diff(r, axis=0), axis=1)
    np.testing.assert_allclose(bonds, b, atol=1e-6)
    dd = r[:, None, :] - r[None, :, :]
    dd -= L * np.floor(dd / L + 0.5)
    dist = np.sqrt((dd ** 2).sum(-1))
    far = np.abs(np.arange(N)[:, None] - np.arange(N)[None, :]) >= 2
    assert dist[far].min() >= rc - 1e-9
    assert np.all(r[2:, 0] >= xw + t - 1 + rc - 1e-9)
    assert np.all(r[2:, 0] <= xw + L[0] - rc + 1e-9)
    solid = np.argwhere(si.solid_mask(p))[:, ::-1].astype(np.float64)
    ds = solid[None, :, :] - np.mod(r[2:, None, :], L)
    ds -= L * np.floor(ds / L + 0.5)
    assert np.sqrt((ds ** 2).sum(-1)).min() >= rc - 1e-9


@pytest.mark.parametrize("which", ["small0", "small1", "ragged100", "paper400"])
def test_seeded_start_is_a_self_avoiding_walk(which):
    lb = _lb()
    p = {"small0": si.small_translocation(0), "small1": si.small_translocation(11),
         "ragged100": si.ragged_member(100, 3, seed=77), "paper400": si.paper_translocation(5)}[which]
    sim = lb.Simulation(p)  # no init_pos
    r, v = sim.beads()
    check_walk(p, r)
    assert np.all(v == 0)
    assert sim.status()["state"] == lb.RUNNING and sim.status()["n_trans"] == 0


def test_seeded_start_depends_on_the_seed_only():
    lb = _lb()
    p = si.small_translocation(3)
    a = lb.Simulation(p).beads()[0]
    b = lb.Simulation(dict(p)).beads()[0]
    np.testing.assert_array_equal(a, b)
    c = lb.Simulation(dict(p, seed=4)).beads()[0]
    assert np.abs(a[2:] - c[2:]).max() > 0.1
    # the same start in another storage type and in an ensemble
    np.testing.assert_array_equal(a, lb.Simulation(dict(p, storage="f16")).beads()[0])
    ens = lb.Ensemble([p, dict(p, seed=4)], [None, None])
    np.testing.assert_array_equal(ens.beads(0)[0], a)
    np.testing.assert_array_equal(ens.beads(1)[0], c)


def test_seeded_start_steps_like_the_oracle():
    lb = _lb()
    p = dict(si.small_translocation(6), lj_eps=2e-3)
    sim = lb.Simulation(p)
    r0 = sim.beads()[0]
    orc = oracle.OracleSim(p, init_pos=r0)
    for n in (1, 9):
        sim.step(n)
        orc.step(n)
    assert rel_err(sim.populations(), orc.populations()) < 2e-5
    assert np.abs(sim.beads()[0] - orc.beads()[0]).max() < 1e-5
    assert sim.status() == orc.status()


def test_seeded_start_rejects_a_box_too_small():
    lb = _lb()
    p = dict(si.small_translocation(0), nx=8, ny=4, nz=4, wall_x=4, pore_d=1, n_beads=30)
    with pytest.raises(lb.LbmdError) as e:
        lb.Simulation(p)
    assert e.value.code == lb.lbmd.LBMD_EINVAL
