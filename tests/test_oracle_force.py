"""Pins of the oracle's symmetric hydro force (Eq. 7) with Monaghan viscosity
and the matching energy equation (Eq. 5).

Conservation laws hold for any correct pairwise-antisymmetric discretisation,
the two-particle values are derived by hand, and brute force must agree with
the cell list bit for bit.
"""
import math

import numpy as np
import pytest

import sph_inputs


def _cloud_state(orc, n, seed):
    wl = sph_inputs.random_cloud(n, seed=seed, vel=0.5)
    x, v, m, h, u = wl.col("x"), wl.col("v"), wl.col("m"), wl.col("h"), wl.col("u")
    d = orc.density(x, m, h, wl.box, wl.eta, wl.h_cap, 3)
    P, c = orc.eos(d["rho"], u, wl.gamma)
    return wl, x, v, m, d["h"], d["rho"], P, c


def test_momentum_conservation(orc):
    wl, x, v, m, h, rho, P, c = _cloud_state(orc, 600, 21)
    f = orc.force(x, v, m, h, rho, P, c, wl.box, 1.0, 2.0, 0.01)
    ma = m[:, None] * f["a"]
    assert np.all(np.abs(ma.sum(0)) <= 1e-12 * np.abs(ma).sum(0))


def test_total_energy_conservation(orc):
    wl, x, v, m, h, rho, P, c = _cloud_state(orc, 600, 22)
    f = orc.force(x, v, m, h, rho, P, c, wl.box, 1.0, 2.0, 0.01)
    kin = m * np.sum(v * f["a"], axis=1)
    th = m * f["dudt"]
    assert abs(kin.sum() + th.sum()) <= 1e-12 * (np.abs(kin).sum() + np.abs(th).sum())
    # the viscosity only heats
    f0 = orc.force(x, v, m, h, rho, np.zeros_like(P), c, wl.box, 1.0, 2.0, 0.01)
    assert f0["dudt"].sum() >= 0.0


def test_uniform_pressure_lattice_has_no_force(orc):
    n, s = 10, 0.1
    i = np.arange(n)
    z, y, xx = np.meshgrid(i, i, i, indexing="ij")
    x = (np.stack([xx.ravel(), y.ravel(), z.ravel()], 1) + 0.5) * s
    N = len(x)
    one = np.ones(N)
    f = orc.force(x, np.zeros((N, 3)), one, np.full(N, 1.3 * s), one, one, one,
                  (1.0, 1.0, 1.0), 1.0, 2.0, 0.01)
    # one pair term is about m (2P/rho^2) |dW/dr| ~ 2 / (pi h^4) ~ 220
    assert np.max(np.abs(f["a"])) < 1e-10
    assert np.max(np.abs(f["dudt"])) == 0.0


def test_two_particles_pressure_only(orc):
    # h_i = h_j = 1, r = 1 on the x axis, m = rho = P = 1, v = 0:
    # grad_i W = x_hat * (1/pi) w'(1) = -0.75/pi x_hat, so
    # a_i = -m (P/rho^2 + P/rho^2) grad_i W = +1.5/pi x_hat (repulsive).
    x = [[3.0, 2.0, 2.0], [2.0, 2.0, 2.0]]
    f = orc.force(x, np.zeros((2, 3)), [1, 1], [1, 1], [1, 1], [1, 1], [1, 1],
                  (10.0, 10.0, 10.0), 1.0, 2.0, 0.01, brute=True)
    assert f["a"][0, 0] == pytest.approx(0.477464829275686, rel=1e-14)
    assert f["a"][1, 0] == pytest.approx(-0.477464829275686, rel=1e-14)
    assert np.all(f["a"][:, 1:] == 0.0)
    assert np.all(f["dudt"] == 0.0)
    assert list(f["nngb"]) == [1, 1]


def test_two_particles_viscosity_only(orc):
    # P = 0, c = 1, rho = 1, m = 1, h = 1, r = 1; i approaches j with v_i = -x_hat.
    # v_ij . r_ij = -1 < 0, mu = h v.r / (r^2 + eps h^2) = -1/1.01,
    # Pi = (-alpha c mu + beta mu^2)/rho = 0.990099.. + 2 * 0.980296.. = 2.95069..,
    # a_i = -m Pi grad_i W = +Pi * 0.75/pi = 0.7044256..,
    # du_i/dt = m (Pi/2) v_ij . grad_i W = (Pi/2)(0.75/pi) = 0.3522128..
    x = [[3.0, 2.0, 2.0], [2.0, 2.0, 2.0]]
    v = [[-1.0, 0.0, 0.0], [0.0, 0.0, 0.0]]
    f = orc.force(x, v, [1, 1], [1, 1], [1, 1], [0, 0], [1, 1], (10.0, 10.0, 10.0),
                  1.0, 2.0, 0.01, brute=True)
    assert f["a"][0, 0] == pytest.approx(0.704425613233906, rel=1e-13)
    assert f["a"][1, 0] == pytest.approx(-0.704425613233906, rel=1e-13)
    assert f["dudt"][0] == pytest.approx(0.352212806616953, rel=1e-13)
    assert f["dudt"][1] == pytest.approx(0.352212806616953, rel=1e-13)
    # receding pair: no viscosity at all
    f2 = orc.force(x, [[1.0, 0, 0], [0, 0, 0]], [1, 1], [1, 1], [1, 1], [0, 0], [1, 1],
                   (10.0, 10.0, 10.0), 1.0, 2.0, 0.01, brute=True)
    assert np.all(f2["a"] == 0.0) and np.all(f2["dudt"] == 0.0)


def test_pair_cutoff_uses_mean_smoothing_length(orc):
    # r < h_i + h_j: with h = (1, 0.5) the pair interacts at r = 1.49, not at 1.51
    for r, expect in ((1.49, 1), (1.51, 0)):
        x = [[2.0 + r, 2.0, 2.0], [2.0, 2.0, 2.0]]
        f = orc.force(x, np.zeros((2, 3)), [1, 1], [1.0, 0.5], [1, 1], [1, 1], [1, 1],
                      (10.0, 10.0, 10.0), 1.0, 2.0, 0.01, brute=True)
        assert list(f["nngb"]) == [expect, expect]


def test_bruteforce_equals_cell_list_bitwise(orc):
    wl, x, v, m, h, rho, P, c = _cloud_state(orc, 500, 23)
    a = orc.force(x, v, m, h, rho, P, c, wl.box, 1.0, 2.0, 0.01, brute=True)
    b = orc.force(x, v, m, h, rho, P, c, wl.box, 1.0, 2.0, 0.01, brute=False)
    for k in ("a", "dudt", "nngb"):
        assert np.array_equal(a[k], b[k]), k


def test_kick_drift_closed_form(orc):
    # constant a and du/dt: after k symplectic-Euler steps
    #   v_k = v0 + k a dt,  x_k = x0 + k v0 dt + a dt^2 k (k+1)/2,  u_k = u0 + k dudt dt
    rng = np.random.default_rng(3)
    n, dt, K = 50, 1e-3, 7
    x0 = rng.uniform(0.3, 0.7, (n, 3))
    v0 = rng.uniform(-1, 1, (n, 3))
    a = rng.uniform(-2, 2, (n, 3))
    u0 = rng.uniform(1, 2, n)
    du = rng.uniform(-1, 1, n)
    x, v, u = x0, v0, u0
    for _ in range(K):
        x, v, u = orc.kick_drift(x, v, a, u, du, dt, dt, (1.0, 1.0, 1.0))
    np.testing.assert_allclose(v, v0 + K * a * dt, rtol=0, atol=1e-14)
    np.testing.assert_allclose(x, x0 + K * v0 * dt + a * dt * dt * K * (K + 1) / 2,
                               rtol=0, atol=1e-14)
    np.testing.assert_allclose(u, u0 + K * du * dt, rtol=0, atol=1e-14)


def test_kick_drift_wraps_periodically(orc):
    x, v, u = orc.kick_drift([[0.99, 0.01, 0.5]], [[0.02, -0.02, 0.0]], np.zeros((1, 3)),
                             [1.0], [0.0], 1.0, 1.0, (1.0, 1.0, 1.0))
    np.testing.assert_allclose(x[0], [0.01, 0.99, 0.5], atol=1e-15)
    assert np.all((x >= 0) & (x < 1))
