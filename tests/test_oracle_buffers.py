"""Pins of the oracle's buffer kernels (the paper's benchmark grouping, Section
6: contiguous buffers of B co-located particles, every pair of a buffer).

Each check ties the buffer functions to something fixed independently of
them: hand-derived closed forms, the full-neighbourhood density and force
(pinned in their own tests) in the case where one buffer holds every particle,
block-diagonal structure, conservation within a buffer, and invariance under
a periodic translation."""
import math

import numpy as np
import pytest

import oracle
import sph_inputs

SIGMA = 1.0 / math.pi


def _blocks(nb=(2, 2, 2), seed=3):
    return sph_inputs.buffer_blocks(nb=nb, seed=seed)


def _cols(wl):
    return (wl.col("x").copy(), wl.col("v").copy(), wl.col("m").copy(), wl.col("h").copy(),
            wl.col("u").copy())


def test_two_particle_buffer_closed_form():
    # two particles at r = h (equal h): w(0) = 1 and w(1) = 1/4, so
    # rho_0 = sigma / h^3 (m_0 + m_1 / 4) and rho_1 = sigma / h^3 (m_1 + m_0 / 4)
    h = 0.1
    x = np.array([[0.3, 0.5, 0.5], [0.4, 0.5, 0.5]])
    m = np.array([2.0, 3.0])
    u = np.array([1.0, 2.0])
    d = oracle.buffer_density(x, m, [h, h], u, (1.0, 1.0, 1.0), 5.0 / 3.0, 64)
    want = SIGMA / h ** 3 * np.array([m[0] + m[1] / 4, m[1] + m[0] / 4])
    assert np.allclose(d["rho"], want, rtol=1e-14)
    assert np.allclose(d["P"], (2.0 / 3.0) * want * u, rtol=1e-14)
    assert np.allclose(d["c"], np.sqrt(5.0 / 3.0 * d["P"] / want), rtol=1e-14)
    assert list(d["nngb"]) == [1, 1]


def test_two_particle_buffer_force_closed_form():
    # pressure only (no relative velocity): a_0 = -m_1 (P0/rho0^2 + P1/rho1^2) grad W,
    # grad_0 W = (x_0 - x_1)/r * sigma / hb^4 * w'(r/hb), w'(1) = -3/4
    h = 0.1
    x = np.array([[0.3, 0.5, 0.5], [0.4, 0.5, 0.5]])
    v = np.zeros((2, 3))
    m = np.array([2.0, 3.0])
    rho = np.array([1.5, 2.5])
    P = np.array([0.7, 0.9])
    c = np.array([1.0, 1.0])
    f = oracle.buffer_force(x, v, m, [h, h], rho, P, c, (1.0, 1.0, 1.0), 1.0, 2.0, 0.01, 64)
    gw = SIGMA / h ** 4 * (-0.75)                      # dW/dr at r = h
    k = P[0] / rho[0] ** 2 + P[1] / rho[1] ** 2
    a0 = -m[1] * k * gw * np.array([-1.0, 0.0, 0.0])   # (x_0 - x_1) / r = -e_x
    a1 = -m[0] * k * gw * np.array([1.0, 0.0, 0.0])
    assert np.allclose(f["a"][0], a0, rtol=1e-13, atol=0)
    assert np.allclose(f["a"][1], a1, rtol=1e-13, atol=0)
    assert np.allclose(f["dudt"], 0.0, atol=1e-15)


def test_one_buffer_equals_full_neighbourhood():
    # with every particle in one buffer and a box much larger than the
    # support, the buffer kernels are the full density (h fixed) and force
    wl = sph_inputs.random_cloud(64, seed=11, box=(1.0, 1.0, 1.0), vel=2.0)
    x, v, m, h, u = _cols(wl)
    x = 0.4 + 0.2 * x                                   # a 0.2-wide cluster in the unit box
    h[:] = 0.05
    d = oracle.buffer_density(x, m, h, u, wl.box, wl.gamma, 64)
    full = oracle.density(x, m, h, wl.box, wl.eta, 1.0, 0, brute=True)
    assert np.allclose(d["rho"], full["rho"], rtol=1e-13, atol=0)
    assert np.array_equal(d["nngb"], full["nngb"])
    P, c = oracle.eos(full["rho"], u, wl.gamma)
    assert np.allclose(d["P"], P, rtol=1e-13) and np.allclose(d["c"], c, rtol=1e-13)
    f = oracle.buffer_force(x, v, m, h, d["rho"], d["P"], d["c"], wl.box, 1.0, 2.0, 0.01, 64)
    ff = oracle.force(x, v, m, h, d["rho"], d["P"], d["c"], wl.box, 1.0, 2.0, 0.01, brute=True)
    scale = np.mean(np.linalg.norm(ff["a"], axis=1))
    assert np.max(np.abs(f["a"] - ff["a"])) <= 1e-12 * scale
    assert np.max(np.abs(f["dudt"] - ff["dudt"])) <= 1e-12 * np.mean(np.abs(ff["dudt"]))
    assert np.array_equal(f["nngb"], ff["nngb"])


def test_buffers_are_independent():
    # changing the particles of buffer 1 leaves buffer 0's results bit for bit
    wl = _blocks()
    B = wl.meta["B"]
    x, v, m, h, u = _cols(wl)
    d0 = oracle.buffer_density(x, m, h, u, wl.box, wl.gamma, B)
    f0 = oracle.buffer_force(x, v, m, h, d0["rho"], d0["P"], d0["c"], wl.box, 1.0, 2.0, 0.01, B)
    rng = np.random.default_rng(1)
    x2, v2 = x.copy(), v.copy()
    x2[B:2 * B] = rng.uniform(0, 1, (B, 3))
    v2[B:2 * B] = rng.uniform(-5, 5, (B, 3))
    d1 = oracle.buffer_density(x2, m, h, u, wl.box, wl.gamma, B)
    f1 = oracle.buffer_force(x2, v2, m, h, d1["rho"], d1["P"], d1["c"], wl.box, 1.0, 2.0, 0.01, B)
    keep = np.r_[0:B, 2 * B:wl.n]
    assert np.array_equal(d0["rho"][keep], d1["rho"][keep])
    assert np.array_equal(f0["a"][keep], f1["a"][keep])
    assert not np.array_equal(d0["rho"][B:2 * B], d1["rho"][B:2 * B])


def test_conservation_within_each_buffer():
    # the pair terms are antisymmetric inside a buffer: momentum and total
    # energy are conserved buffer by buffer
    wl = _blocks(seed=4)
    B = wl.meta["B"]
    x, v, m, h, u = _cols(wl)
    d = oracle.buffer_density(x, m, h, u, wl.box, wl.gamma, B)
    f = oracle.buffer_force(x, v, m, h, d["rho"], d["P"], d["c"], wl.box, 1.0, 2.0, 0.01, B)
    for b in range(wl.n // B):
        sl = slice(b * B, (b + 1) * B)
        ma = m[sl, None] * f["a"][sl]
        scale = np.sum(np.abs(ma))
        assert np.all(np.abs(ma.sum(axis=0)) <= 1e-12 * scale)
        e = m[sl] * (np.sum(v[sl] * f["a"][sl], axis=1) + f["dudt"][sl])
        assert abs(e.sum()) <= 1e-12 * np.sum(np.abs(m[sl] * f["dudt"][sl]))


def test_periodic_translation_invariance():
    # shifting every particle by half the box (wrapped) changes no result
    # beyond rounding: separations are minimum images
    wl = _blocks(seed=5)
    B = wl.meta["B"]
    x, v, m, h, u = _cols(wl)
    box = np.asarray(wl.box)
    xs = (x + 0.5 * box) % box
    d0 = oracle.buffer_density(x, m, h, u, box, wl.gamma, B)
    d1 = oracle.buffer_density(xs, m, h, u, box, wl.gamma, B)
    assert np.allclose(d0["rho"], d1["rho"], rtol=1e-12)
    f0 = oracle.buffer_force(x, v, m, h, d0["rho"], d0["P"], d0["c"], box, 1.0, 2.0, 0.01, B)
    f1 = oracle.buffer_force(xs, v, m, h, d0["rho"], d0["P"], d0["c"], box, 1.0, 2.0, 0.01, B)
    scale = np.mean(np.linalg.norm(f0["a"], axis=1))
    assert np.max(np.abs(f0["a"] - f1["a"])) <= 1e-10 * scale


@pytest.mark.parametrize("tail", [1, 5, 63])
def test_ragged_last_buffer(tail):
    # the last buffer holds n mod B particles and sees only them
    wl = _blocks(seed=6)
    B = wl.meta["B"]
    n = 2 * B + tail
    x, v, m, h, u = (a[:n] for a in _cols(wl))
    d = oracle.buffer_density(x, m, h, u, wl.box, wl.gamma, B)
    d_tail = oracle.buffer_density(x[2 * B:], m[2 * B:], h[2 * B:], u[2 * B:], wl.box, wl.gamma, B)
    assert np.array_equal(d["rho"][2 * B:], d_tail["rho"])
    f = oracle.buffer_force(x, v, m, h, d["rho"], d["P"], d["c"], wl.box, 1.0, 2.0, 0.01, B)
    f_tail = oracle.buffer_force(x[2 * B:], v[2 * B:], m[2 * B:], h[2 * B:], d_tail["rho"], d_tail["P"],
                                 d_tail["c"], wl.box, 1.0, 2.0, 0.01, B)
    assert np.array_equal(f["a"][2 * B:], f_tail["a"])


def test_lattice_block_density_matches_direct_sum():
    # an exact 4x4x4 block (no jitter) of spacing s, h = 1.2 s: the corner
    # particle's density is the direct sum over the 64 lattice sites, written
    # out with the spline pieces
    s, hh = 0.01, 0.012
    g = np.arange(4) * s + 0.5
    x = np.array([[a, b, c] for c in g for b in g for a in g])
    m = np.full(64, 1.0)
    d = oracle.buffer_density(x, m, np.full(64, hh), np.ones(64), (1.0, 1.0, 1.0), 5.0 / 3.0, 64)

    def w(q):
        if q < 1.0:
            return 1.0 - 1.5 * q * q + 0.75 * q ** 3
        if q < 2.0:
            return 0.25 * (2.0 - q) ** 3
        return 0.0
    want = sum(w(math.sqrt(i * i + j * j + k * k) * s / hh)
               for i in range(4) for j in range(4) for k in range(4)) * SIGMA / hh ** 3
    assert d["rho"][0] == pytest.approx(want, rel=1e-13)


def test_buffer_relative_offsets():
    # offsets from the buffer's first particle, moved to the nearest image:
    # a block straddling the periodic boundary gets small offsets, and origin
    # plus offset is the position modulo the box
    wl = _blocks(seed=7)
    B = wl.meta["B"]
    x = wl.col("x")
    box = np.asarray(wl.box)
    origin, off = oracle.buffer_relative(x, box, B, "fp32")
    assert np.all(np.abs(off) < 0.5 * box)
    assert np.max(np.abs(off)) < 5 * wl.meta["spacing"]
    back = (origin + off) % box
    err = np.abs(back - x)
    err = np.minimum(err, box - err)
    assert np.max(err) <= 4e-7 * np.max(np.abs(off)) + 1e-15
    assert np.array_equal(origin[::B], x[::B]) and np.all(off[::B] == 0.0)
