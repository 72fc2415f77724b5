"""Pins of the oracle's lattice-Boltzmann part (Sec. II, Eqs. 5-10) against
what the mathematics fixes: lattice isotropy, equilibrium moments, the
collision fixed point, exact conservation, source moments, a brute-force
re-implementation on tiny boxes, the Poiseuille curvature and the Taylor-Green
decay rate given by nu = c_s^2 (tau - 1/2)."""
import itertools
import math

import numpy as np
import pytest

import oracle
import seeded_inputs as si

CS2 = 1.0 / 3.0


def test_lattice_isotropy():
    """The D3Q19 set with weights 1/3, 1/18, 1/36 is isotropic to fourth order
    (needed for Eq. 6 to give Navier-Stokes): sum w = 1, sum w c = 0,
    sum w c c = c_s^2 I, sum w cccc = c_s^4 (dd + dd + dd)."""
    w, c = oracle.lattice()
    c = c.astype(float)
    assert abs(w.sum() - 1) < 1e-15
    assert np.abs(np.einsum("p,pa->a", w, c)).max() < 1e-15
    np.testing.assert_allclose(np.einsum("p,pa,pb->ab", w, c, c), CS2 * np.eye(3), atol=1e-15)
    assert np.abs(np.einsum("p,pa,pb,pc->abc", w, c, c, c)).max() < 1e-15
    d = np.eye(3)
    iso4 = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                       + np.einsum("ad,bc->abcd", d, d))
    np.testing.assert_allclose(np.einsum("p,pa,pb,pc,pd->abcd", w, c, c, c, c), iso4, atol=1e-15)
    # opposite directions adjacent: c_{2k} = -c_{2k-1}
    for p in range(1, 19, 2):
        assert np.all(c[p] == -c[p + 1])
    assert len({tuple(v) for v in c}) == 19


def test_equilibrium_moments():
    """Eqs. 6-9: the equilibrium carries density rho, momentum rho u and
    momentum flux rho c_s^2 I + rho u u."""
    rng = np.random.default_rng(1)
    w, c = oracle.lattice()
    c = c.astype(float)
    for _ in range(20):
        rho = rng.uniform(0.8, 1.2)
        u = rng.uniform(-0.1, 0.1, 3)
        f = oracle.equilibrium(rho, u)
        assert abs(f.sum() - rho) < 1e-14
        np.testing.assert_allclose(f @ c, rho * u, atol=1e-15)
        P = np.einsum("p,pa,pb->ab", f, c, c)
        np.testing.assert_allclose(P, rho * CS2 * np.eye(3) + rho * np.outer(u, u), atol=1e-15)
    # Eq. 6 written with the full tensor contraction uu:(cc - c_s^2 I)
    rho, u = 1.07, np.array([0.03, -0.02, 0.05])
    ref = np.array([w[p] * rho * (1 + c[p] @ u / CS2 + np.einsum("ab,ab->", np.outer(u, u),
                   np.outer(c[p], c[p]) - CS2 * np.eye(3)) / (2 * CS2 ** 2)) for p in range(19)])
    np.testing.assert_allclose(oracle.equilibrium(rho, u), ref, rtol=1e-14, atol=0)


def test_collision_fixed_point():
    """P1: f = f_eq(rho, u) is unchanged by the BGK collision without forcing."""
    rng = np.random.default_rng(2)
    for tau in (0.51, 0.6, 0.8, 1.0, 1.7):
        for _ in range(10):
            f = oracle.equilibrium(rng.uniform(0.9, 1.1), rng.uniform(-0.057, 0.057, 3))
            np.testing.assert_allclose(oracle.collide(f, tau), f, rtol=0, atol=1e-15)


def test_collision_conserves_and_relaxes():
    """Eq. 5: collision keeps rho and rho u, relaxes the non-equilibrium part
    by (1 - 1/tau), and tau = 1 lands exactly on f_eq."""
    rng = np.random.default_rng(3)
    w, c = oracle.lattice()
    for tau in (0.6, 1.0, 1.4):
        f = oracle.equilibrium(1.0, [0.02, 0.01, -0.03]) * (1 + 0.05 * rng.standard_normal(19))
        out = oracle.collide(f, tau)
        assert abs(out.sum() - f.sum()) < 1e-15
        np.testing.assert_allclose(out @ c, f @ c, atol=1e-16)
        rho, u = oracle.moments(f)
        feq = oracle.equilibrium(rho, u)
        np.testing.assert_allclose(out - feq, (1 - 1 / tau) * (f - feq), atol=1e-16)


def test_source_moments():
    """P3: the source of Eq. 10 injects no mass and exactly the force as
    momentum; with the Guo flag the body force g also adds exactly g to the
    momentum of one collision."""
    rng = np.random.default_rng(4)
    w, c = oracle.lattice()
    for forcing in ("paper", "guo"):
        for tau in (0.6, 1.0):
            f = oracle.equilibrium(1.0, [0.01, 0.0, 0.02]) * (1 + 0.02 * rng.standard_normal(19))
            Fb = rng.uniform(-1e-3, 1e-3, 3)
            g = rng.uniform(-1e-3, 1e-3, 3)
            out = oracle.collide(f, tau, Fb=Fb, g=g, forcing=forcing)
            assert abs(out.sum() - f.sum()) < 1e-15
            np.testing.assert_allclose(out @ c - f @ c, Fb + g, atol=1e-17)


def test_guo_source_second_moment():
    """Guo et al. (2002): the second-order source carries zero mass, momentum
    (1 - 1/(2 tau)) g and momentum flux (1 - 1/(2 tau)) (u g + g u), which is
    what cancels the discrete-lattice error of the body force."""
    rng = np.random.default_rng(14)
    w, c = oracle.lattice()
    c = c.astype(float)
    for tau in (0.6, 1.3):
        f = oracle.equilibrium(1.0, rng.uniform(-0.05, 0.05, 3))
        g = rng.uniform(-1e-3, 1e-3, 3)
        rho, u = oracle.moments(f, g, "guo")
        # source = collide(f) - BGK part; f is an equilibrium of its unshifted u,
        # so isolate the source by subtracting the collision without force
        src = oracle.collide(f, tau, g=g, forcing="guo") - (
            f - (f - oracle.equilibrium(rho, u)) / tau)
        k = 1 - 0.5 / tau
        assert abs(src.sum()) < 1e-16
        np.testing.assert_allclose(src @ c, k * g, atol=1e-16)
        np.testing.assert_allclose(np.einsum("p,pa,pb->ab", src, c, c),
                                   k * (np.outer(u, g) + np.outer(g, u)), atol=1e-16)


# -- brute force on tiny boxes (P10) ------------------------------------------

def _brute_force_step(f, solid, tau, g, forcing, F):
    """Independent one-step LB update written from Eqs. 5-8 and 10 with plain
    loops: moments, equilibrium by the full tensor contraction, source, then
    *pull* streaming with halfway bounce-back (the oracle pushes)."""
    w, c = oracle.lattice()
    c = c.astype(float)
    nz, ny, nx = solid.shape
    opp = [0] + [p + 1 if p % 2 == 1 else p - 1 for p in range(1, 19)]
    post = np.zeros_like(f)
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        if solid[z, y, x]:
            continue
        fl = f[:, z, y, x]
        rho = sum(fl)
        mom = sum(fl[p] * c[p] for p in range(19))
        if forcing == "guo":
            mom = mom + 0.5 * np.asarray(g)
        u = mom / rho
        for p in range(19):
            feq = w[p] * rho * (1 + c[p] @ u / CS2 + np.einsum(
                "ab,ab->", np.outer(u, u), np.outer(c[p], c[p]) - CS2 * np.eye(3)) / (2 * CS2 ** 2))
            Fx = F[:, z, y, x]
            src = w[p] / CS2 * (c[p] @ Fx)
            if forcing == "guo":
                src += (1 - 0.5 / tau) * w[p] * (((c[p] - u) / CS2 + (c[p] @ u) * c[p] / CS2 ** 2) @ g)
            else:
                src += w[p] / CS2 * (c[p] @ g)
            post[p, z, y, x] = fl[p] - (fl[p] - feq) / tau + src
    new = np.zeros_like(f)
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        if solid[z, y, x]:
            continue
        for p in range(19):
            xs, ys, zs = (x - int(c[p][0])) % nx, (y - int(c[p][1])) % ny, (z - int(c[p][2])) % nz
            if solid[zs, ys, xs]:
                new[p, z, y, x] = post[opp[p], z, y, x]
            else:
                new[p, z, y, x] = post[p, zs, ys, xs]
    return new


@pytest.mark.parametrize("shape,wall,ywalls,forcing", [
    ((4, 4, 4), (2, 2, 1, 1), 0, "paper"),
    ((4, 4, 4), (1, 1, 0, 2), 1, "guo"),
    ((5, 4, 3), (3, 1, 1, 1), 0, "paper"),
    ((3, 5, 4), (-1, 1, 0, 0), 1, "guo"),
])
def test_brute_force_tiny_box(shape, wall, ywalls, forcing):
    nx, ny, nz = shape
    wall_x, thick, pore_d, pore_y0 = wall
    p = dict(nx=nx, ny=ny, nz=nz, wall_x=wall_x, wall_thickness=thick, pore_d=pore_d,
             pore_y0=pore_y0, pore_z0=0, y_walls=ywalls, tau=0.7, forcing=forcing,
             body_force=(1e-3, -2e-3, 5e-4))
    rho0, u0 = si.random_flow((nz, ny, nx), seed=11, u_max=0.05)
    s = oracle.OracleSim(p, init_rho=rho0, init_u=u0)
    f0 = s.populations()
    solid = s.solid().astype(bool)
    assert np.all(f0[:, solid] == 0)
    for n in range(3):
        s.step(1)
        ref = _brute_force_step(f0, solid, p["tau"], np.array(p["body_force"]), forcing,
                                np.zeros((3, nz, ny, nx)))
        np.testing.assert_allclose(s.populations(), ref, rtol=1e-13, atol=1e-15)
        f0 = ref


def test_brute_force_with_bead_force():
    """The bead force field enters the collision exactly as Eq. 10's source."""
    p = dict(si.small_translocation(3, n_beads=3))
    p.update(nx=8, ny=8, nz=8, wall_x=1, pore_d=3, lj_sigma=0.6, kT=1e-3)
    pos = np.array([[5.3, 2.1 + 1.2 * i, 4.2 + 0.1 * i] for i in range(3)])
    pos[:, 2] = 4.2
    pos[2] = pos[1] + 1.2 * np.array([0.6, 0.8, 0.0])
    s = oracle.OracleSim(p, init_pos=pos)
    f0 = s.populations()
    s.step(1)
    F = s.force_field()
    assert np.abs(F).max() > 0
    ref = _brute_force_step(f0, s.solid().astype(bool), 1.0, np.zeros(3), "paper", F)
    np.testing.assert_allclose(s.populations(), ref, rtol=1e-13, atol=1e-16)


def test_rest_state_is_stationary_with_walls():
    p = dict(si.small_translocation(0, n_beads=0))
    p.update(y_walls=1)
    s = oracle.OracleSim(p)
    f0 = s.populations()
    s.step(5)
    np.testing.assert_allclose(s.populations(), f0, rtol=0, atol=1e-15)


def test_mass_and_momentum_conservation_periodic():
    """P2: periodic box, no force: sum f and sum f c are constant to round-off."""
    p = dict(nx=8, ny=6, nz=5, wall_x=-1, tau=0.8)
    rho0, u0 = si.random_flow((5, 6, 8), seed=5, u_max=0.05)
    s = oracle.OracleSim(p, init_rho=rho0, init_u=u0)
    w, c = oracle.lattice()
    f = s.populations()
    m0, P0 = f.sum(), np.einsum("pzyx,pa->a", f, c)
    for _ in range(10):
        s.step(20)
        f = s.populations()
        assert abs(f.sum() - m0) / m0 < 1e-13
        np.testing.assert_allclose(np.einsum("pzyx,pa->a", f, c), P0, atol=1e-12)


def test_bounce_back_conserves_mass():
    p = dict(si.small_translocation(0, n_beads=0))
    p.update(y_walls=1, tau=0.7)
    rho0, u0 = si.random_flow((16, 16, 32), seed=6, u_max=0.03)
    s = oracle.OracleSim(p, init_rho=rho0, init_u=u0)
    m0 = s.populations().sum()
    s.step(50)
    assert abs(s.populations().sum() - m0) / m0 < 1e-13


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.0])
def test_poiseuille_curvature(tau):
    """P5: steady channel flow under body force g has u_x'' = -g / (rho nu) with
    nu = c_s^2 (tau - 1/2) (Sec. II viscosity relation); BGK reproduces the
    parabola exactly at steady state."""
    g = 1e-6
    p = dict(nx=1, ny=34, nz=1, y_walls=1, wall_x=-1, tau=tau, body_force=(g, 0, 0))
    s = oracle.OracleSim(p)
    s.step(80000)
    rho, u = s.fields()
    ux = u[0, 0, :, 0]
    nu = CS2 * (tau - 0.5)
    y = np.arange(1, 33)
    curv = 2 * np.polyfit(y, ux[1:33], 2)[0]
    assert abs(curv / (-g / nu) - 1) < 1e-6
    d2 = ux[1:31] - 2 * ux[2:32] + ux[3:33]
    assert np.abs(d2 / (-g / nu) - 1).max() < 1e-6


def test_poiseuille_magic_tau_zero_slip():
    """P5: with second-order (Guo) forcing and tau = 1/2 + sqrt(3)/4, i.e. the
    TRT 'magic' parameter Lambda = 3/16, halfway bounce-back puts the no-slip
    wall exactly half a node off the solid row."""
    tau = 0.5 + math.sqrt(3) / 4
    p = dict(nx=1, ny=34, nz=1, y_walls=1, wall_x=-1, tau=tau, body_force=(1e-6, 0, 0),
             forcing="guo")
    s = oracle.OracleSim(p)
    s.step(80000)
    rho, u = s.fields()
    c = np.polyfit(np.arange(1, 33), u[0, 0, 1:33, 0], 2)
    r = np.sort(np.roots(c).real)
    np.testing.assert_allclose(r, [0.5, 32.5], atol=1e-6)


@pytest.mark.parametrize("tau", [0.6, 1.0])
def test_taylor_green_decay(tau):
    """P6: a 2-D Taylor-Green vortex (L = 64, A = 0.01) decays as exp(-2 nu k^2 t)."""
    L, A = 64, 0.01
    s = oracle.OracleSim(dict(nx=L, ny=L, nz=1, wall_x=-1, tau=tau),
                         init_u=si.taylor_green_field(L, L, 1, A))
    k = 2 * math.pi / L
    x = np.arange(L)[None, :]
    y = np.arange(L)[:, None]
    basis = np.sin(k * x) * np.cos(k * y)
    ts, amps = [], []
    for n in range(0, 2001, 100):
        if n:
            s.step(100)
        if n >= 500:
            u = s.fields()[1]
            ts.append(n)
            amps.append((u[0, 0] * basis).sum() / (basis * basis).sum())
    rate = -np.polyfit(ts, np.log(amps), 1)[0]
    nu = CS2 * (tau - 0.5)
    assert abs(rate / (2 * nu * k * k) - 1) < 1e-3
