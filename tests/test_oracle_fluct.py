"""Pins of the oracle's thermal source F_p of Eq. 5 (fluctuating LB): a
weight-orthogonal mode basis, noise that leaves mass and momentum untouched,
independent unit normals per non-conserved mode, and -- independently of how
the noise is built -- equipartition of the fluid's momentum and density
fluctuations, <j_a^2> = rho kT and <drho^2> = rho kT / c_s^2 per node, which
the fluctuation-dissipation theorem requires."""
import numpy as np
import pytest

import oracle


def test_mode_basis_is_weight_orthogonal_and_complete():
    e, b = oracle.mode_basis()
    w, c = oracle.lattice()
    G = (e * w[None, :]) @ e.T
    assert np.abs(G - np.diag(np.diag(G))).max() < 1e-15
    assert np.allclose(np.diag(G), b, rtol=1e-15)
    assert np.linalg.matrix_rank(e) == 19
    # the first four rows are the conserved density and momentum
    assert np.array_equal(e[0], np.ones(19)) and np.array_equal(e[1:4].T, c)


def test_noise_conserves_mass_and_momentum():
    w, c = oracle.lattice()
    for node, step in ((0, 0), (12345, 7), (2 ** 31 + 5, 2 ** 33 + 1)):
        xi = oracle.fluct_noise(11, node, step, rho=1.03, tau=0.8, kT=1e-4)
        scale = np.abs(xi).max()
        assert scale > 0
        assert abs(xi.sum()) < 1e-14 * scale
        assert np.abs(c.T @ xi).max() < 1e-14 * scale


def test_noise_mode_variances_and_independence():
    tau, kT, rho = 0.8, 1e-4, 1.0
    e, b = oracle.mode_basis()
    n = 6000
    m = np.array([e @ oracle.fluct_noise(5, node, 3, rho, tau, kT) for node in range(n)])
    g = 1.0 - 1.0 / tau
    var = m.var(axis=0)
    target = 3.0 * rho * kT * b * (1.0 - g * g)  # mu b_k (1 - gamma^2), mu = rho kT / c_s^2
    assert np.all(var[:4] < 1e-30)
    # sample variance of n normals: relative standard error sqrt(2 / n) = 1.8 %
    assert np.all(np.abs(var[4:] / target[4:] - 1.0) < 5 * np.sqrt(2.0 / n))
    corr = np.corrcoef(m[:, 4:].T)
    assert np.abs(corr - np.eye(15)).max() < 5 / np.sqrt(n)


@pytest.mark.parametrize("tau", [0.8, 1.0])
def test_equipartition_of_momentum_and_density(tau):
    kT, n = 1e-4, 12
    p = dict(nx=n, ny=n, nz=n, wall_x=-1, tau=tau, kT_fluid=kT, seed=17)
    s = oracle.OracleSim(p)
    s.step(300)
    j2, d2 = [], []
    for _ in range(40):
        s.step(10)
        rho, u = s.fields()
        j = rho[None] * u
        j2.append((j ** 2).mean())
        d2.append(((rho - 1.0) ** 2).mean())
    # the total momentum and mass are conserved (the k = 0 mode does not
    # fluctuate): factor (1 - 1/V); statistical error of 40 x 1728 x 3 samples
    # of correlated nodes, bound 5 %
    V = n ** 3
    assert np.mean(j2) / (kT * (1 - 1 / V)) == pytest.approx(1.0, abs=0.05)
    assert np.mean(d2) / (3 * kT * (1 - 1 / V)) == pytest.approx(1.0, abs=0.05)
