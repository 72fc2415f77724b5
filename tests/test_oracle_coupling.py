"""Pins of the oracle's grid <-> bead transfer (Sec. II, Fig. 1, Eq. 10):
trilinear interpolation is exact for affine fields, spreading is the negative
adjoint of gathering, and the coupled system conserves fluid + bead momentum."""
import numpy as np
import pytest

import oracle
import seeded_inputs as si


def _affine_field(shape, A, b):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    X = np.stack([x, y, z]).astype(float)  # (3, nz, ny, nx)
    return np.einsum("ab,bzyx->azyx", A, X) + b[:, None, None, None]


def test_trilinear_exact_for_affine_field():
    """P7: with f = f_eq(1, u(x)) the moments return u exactly and trilinear
    interpolation reproduces an affine u at any interior point."""
    shape = (10, 9, 12)
    rng = np.random.default_rng(7)
    A = rng.uniform(-2e-3, 2e-3, (3, 3))
    b = rng.uniform(-0.01, 0.01, 3)
    U = _affine_field(shape, A, b)
    p = dict(nx=12, ny=9, nz=10, wall_x=-1, n_beads=50)
    pos = np.column_stack([rng.uniform(0, 10.99, 50), rng.uniform(0, 7.99, 50), rng.uniform(0, 8.99, 50)])
    s = oracle.OracleSim(p, init_pos=pos, init_u=U, bonds=(np.zeros(0), np.zeros(0), np.zeros(0)))
    ui = s.gather(pos)
    np.testing.assert_allclose(ui, pos @ A.T + b, rtol=0, atol=1e-15)


def test_weights_sum_to_one_and_skip_solids():
    p = si.small_translocation(0, n_beads=1)
    s = oracle.OracleSim(p, init_pos=np.array([[17.0, 7.0, 7.0]]))
    solid = s.solid().reshape(-1)
    rng = np.random.default_rng(8)
    for r in rng.uniform([10, 0, 0], [22, 16, 16], (200, 3)):
        node, w = s.transfer_weights(r)
        assert len(node) >= 4  # a one-node wall can block at most four corners
        assert abs(w.sum() - 1) < 1e-14
        assert np.all(w >= 0)
        assert not np.any(solid[node])
    # all eight corners fluid: weights are the plain trilinear products
    node, w = s.transfer_weights(np.array([20.25, 3.5, 9.75]))
    assert len(node) == 8
    np.testing.assert_allclose(np.sort(w), np.sort(np.outer(np.outer([0.75, 0.25], [0.5, 0.5]),
                                                             [0.25, 0.75]).ravel()), atol=1e-16)


def test_nearest_grid_point():
    p = dict(si.small_translocation(0, n_beads=1), coupling="ngp")
    s = oracle.OracleSim(p, init_pos=np.array([[20.0, 7.0, 7.0]]))
    node, w = s.transfer_weights(np.array([20.49, 3.51, 31.7]))
    assert len(node) == 1 and w[0] == 1.0
    assert node[0] == (0 * 16 + 4) * 32 + 20  # (x, y, z) = (20, 4, 0): z = 31.7 wraps to 15.7, rounds to 16 = 0


def test_ngp_wraps_periodically():
    p = dict(si.small_translocation(0, n_beads=1), coupling="ngp")
    s = oracle.OracleSim(p, init_pos=np.array([[20.0, 7.0, 7.0]]))
    node, _ = s.transfer_weights(np.array([31.6, 15.5, -0.4]))
    assert node[0] == (0 * 16 + 0) * 32 + 0


def test_spread_is_negative_adjoint_of_gather():
    """Eq. 10 with the reaction sign: for any grid field U and bead impulses J,
    sum_x F(x).U(x) = -sum_i J_i . U(r_i), and sum_x F = -sum_i J_i."""
    p = si.small_translocation(0, n_beads=30)
    rng = np.random.default_rng(9)
    pos = si.saw_chain(p, 4)
    U = rng.uniform(-0.05, 0.05, (3, 16, 16, 32))
    s = oracle.OracleSim(p, init_pos=pos, init_u=U)
    solid = s.solid().astype(bool)
    Ug = s.fields()[1]  # the moment field equals U at fluid nodes
    np.testing.assert_allclose(Ug[:, ~solid], U[:, ~solid], atol=1e-15)
    J = rng.standard_normal((30, 3))
    F = s.spread(pos, J)
    assert np.all(F[:, solid] == 0)
    np.testing.assert_allclose(F.reshape(3, -1).sum(1), -J.sum(0), atol=1e-13)
    lhs = np.einsum("azyx,azyx->", F, Ug)
    rhs = -np.einsum("ia,ia->", J, s.gather(pos))
    assert abs(lhs - rhs) < 1e-14


@pytest.mark.parametrize("coupling", ["trilinear", "ngp"])
def test_coupled_momentum_conservation(coupling):
    """P4: periodic box without wall or body force, LJ + bending + noise on:
    fluid momentum (pre-collision sum f c) plus bead momentum sum m v is
    conserved every LB step."""
    p = dict(si.small_translocation(0, n_beads=12))
    p.update(nx=16, ny=12, nz=12, wall_x=-1, pore_d=0, kappa_phi=0.05, kT=1e-3, gamma=0.3,
             coupling=coupling, seed=77)
    pos = si.saw_chain(dict(p, wall_x=-1), 5)
    vel = np.random.default_rng(10).normal(0, 0.02, pos.shape)
    rho0, u0 = si.random_flow((12, 12, 16), seed=12, rho_spread=0.01, u_max=0.01)
    s = oracle.OracleSim(p, init_pos=pos, init_vel=vel, init_rho=rho0, init_u=u0)
    w, c = oracle.lattice()

    def total():
        f = s.populations()
        return np.einsum("pzyx,pa->a", f, c) + p["bead_mass"] * s.beads()[1].sum(0)

    P0 = total()
    for _ in range(25):
        assert s.step(1) == 0
        np.testing.assert_allclose(total(), P0, rtol=0, atol=1e-12)  # round-off of ~4e4 population sums
    # the beads did exchange momentum with the fluid
    assert np.abs(s.bead_aux()[1]).max() > 1e-6
