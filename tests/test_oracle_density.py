"""Pins of the oracle's density sum (Eq. 6) and smoothing-length iteration.

Each check uses a fact fixed outside the oracle's own code: closed forms for
one and two particles, the lattice sum enumerated independently over Z^3,
brute force against the cell list, and a bisection root of the h equation.
"""
import math

import numpy as np
import pytest

import sph_inputs


def test_single_particle_closed_form(orc):
    # one particle: rho = m W(0, h) = m / (pi h^3), no neighbours
    d = orc.density([[0.5, 0.5, 0.5]], [2.0], [0.1], (1.0, 1.0, 1.0), sph_inputs.ETA, 0.2, 0,
                    brute=True)
    assert d["rho"][0] == pytest.approx(2.0 / (math.pi * 0.1 ** 3), rel=1e-15)
    assert d["nngb"][0] == 0


@pytest.mark.parametrize("q,wq", [(1.0, 0.25), (1.5, 0.03125), (0.5, 0.71875)])
def test_two_particles_closed_form(orc, q, wq):
    # rho_i = m/(pi h^3) (w(0) + w(q)); w values by hand:
    #   w(1) = 1 - 1.5 + 0.75 = 0.25;  w(1.5) = 0.25 * 0.5^3;  w(0.5) = 1 - 0.375 + 0.09375
    h = 0.05
    x = [[0.3, 0.4, 0.5], [0.3 + q * h, 0.4, 0.5]]
    d = orc.density(x, [1.0, 1.0], [h, h], (1.0, 1.0, 1.0), sph_inputs.ETA, h, 0, brute=True)
    expect = (1.0 + wq) / (math.pi * h ** 3)
    assert d["rho"][0] == pytest.approx(expect, rel=1e-14)
    assert d["rho"][1] == pytest.approx(expect, rel=1e-14)
    assert list(d["nngb"]) == [1, 1]


def _lattice(n, s):
    i = np.arange(n)
    z, y, x = np.meshgrid(i, i, i, indexing="ij")
    return (np.stack([x.ravel(), y.ravel(), z.ravel()], 1) + 0.5) * s


def _lattice_sum(orc, s, h, m):
    """m * sum over k in Z^3 with |k| s < 2h of W(|k| s, h), and the count of
    k != 0 inside the sphere (integer enumeration)."""
    kmax = int(math.ceil(2 * h / s)) + 1
    rng = np.arange(-kmax, kmax + 1)
    kz, ky, kx = np.meshgrid(rng, rng, rng, indexing="ij")
    k2 = (kx ** 2 + ky ** 2 + kz ** 2).ravel()
    inside = k2 * s * s < 4 * h * h
    r = np.sqrt(k2[inside].astype(np.float64)) * s
    return m * sum(orc.W(ri, h) for ri in r), int(np.count_nonzero(inside)) - 1


@pytest.mark.parametrize("ratio", [1.05, 1.2, 1.3, 1.6])
def test_perfect_lattice_closed_form(orc, ratio):
    n, s, m = 12, 1.0 / 12, 0.37
    h = ratio * s
    x = _lattice(n, s)
    d = orc.density(x, np.full(len(x), m), np.full(len(x), h), (1.0, 1.0, 1.0),
                    sph_inputs.ETA, h, 0)
    expect, cnt = _lattice_sum(orc, s, h, m)
    np.testing.assert_allclose(d["rho"], expect, rtol=1e-13)
    assert np.all(d["nngb"] == cnt)


def test_bruteforce_equals_cell_list_bitwise(orc):
    wl = sph_inputs.random_cloud(700, seed=11)
    x, m, h = wl.col("x"), wl.col("m"), wl.col("h")
    for ns in (0, 3):
        a = orc.density(x, m, h, wl.box, wl.eta, wl.h_cap, ns, brute=True)
        b = orc.density(x, m, h, wl.box, wl.eta, wl.h_cap, ns, brute=False)
        for k in ("rho", "h", "nngb", "drho_dh"):
            assert np.array_equal(a[k], b[k]), k


def test_targets_match_full_run(orc):
    wl = sph_inputs.random_cloud(900, seed=12)
    x, m, h = wl.col("x"), wl.col("m"), wl.col("h")
    full = orc.density(x, m, h, wl.box, wl.eta, wl.h_cap, 5)
    t = np.array([3, 100, 899, 0, 450])
    part = orc.density(x, m, h, wl.box, wl.eta, wl.h_cap, 5, targets=t)
    assert np.array_equal(part["rho"], full["rho"][t])
    assert np.array_equal(part["h"], full["h"][t])


def test_newton_reaches_bisection_root(orc):
    # Root of f(h) = rho(h) - m (eta/h)^3 on a jittered lattice, found by
    # bisection over fixed-h density sums, must equal the Newton iterate.
    wl = sph_inputs.sod(n_lattice=16, seed=5)
    x, m, h0 = wl.col("x"), wl.col("m"), wl.col("h")
    t = np.array([7, 300, 1500, 2100])
    newt = orc.density(x, m, h0, wl.box, wl.eta, wl.h_cap, 5, targets=t)
    for k, i in enumerate(t):
        def f(hh):
            d = orc.density(x, m, np.full(len(x), hh), wl.box, wl.eta, wl.h_cap, 0,
                            targets=[i])
            return d["rho"][0] - m[i] * (wl.eta / hh) ** 3
        lo, hi = 0.5 * h0[i], min(2.0 * h0[i], wl.h_cap)
        assert f(lo) < 0 < f(hi)
        for _ in range(80):
            mid = 0.5 * (lo + hi)
            if f(mid) < 0:
                lo = mid
            else:
                hi = mid
        assert newt["h"][k] == pytest.approx(0.5 * (lo + hi), rel=1e-10)
        rho_fp = m[i] * (wl.eta / newt["h"][k]) ** 3
        assert newt["rho"][k] == pytest.approx(rho_fp, rel=1e-9)


def test_newton_fixed_point_gives_48_neighbours_in_the_continuum(orc):
    # h = eta (m/rho)^(1/3) with eta = 1/2 (3*48/(4 pi))^(1/3) puts 48 particles
    # in the support sphere of a uniform medium: (4 pi/3)(2h)^3 rho/m = 48.
    wl = sph_inputs.sod(n_lattice=20, seed=6)
    d = orc.density(wl.col("x"), wl.col("m"), wl.col("h"), wl.box, wl.eta, wl.h_cap, 5,
                    targets=np.arange(0, 200))
    vol = 4.0 / 3.0 * math.pi * (2 * d["h"]) ** 3
    mean_count = np.mean(vol * d["rho"] / wl.col("m")[:200])
    assert mean_count == pytest.approx(48.0, rel=1e-9)
    assert 35 <= np.mean(d["nngb"]) <= 60


def test_h_cap_clamps_and_flags(orc):
    wl = sph_inputs.random_cloud(300, seed=13, n_ngb=30)
    cap = 0.9 * wl.meta["h"]
    d = orc.density(wl.col("x"), wl.col("m"), wl.col("h"), wl.box, wl.eta, cap, 5)
    assert np.all(d["h"] <= cap)
    assert np.any(d["flags"] & orc.FLAG_HCAP)
