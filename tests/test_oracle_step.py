"""Pins of the oracle's sampled composition ``oracle.step(wl, targets=t)``.

The full-size parity tests evaluate the oracle on a sample of target
particles: the density with its Newton steps on every particle within
2 h_cap of a target (all that a target's force can touch, since h_i + h_j
<= 2 h_cap), then the force on the targets alone.  Each particle's density
sum and force sum are independent of which other particles are evaluated,
so the sampled rows must equal the rows of the whole-set step bit for bit;
a ball too small, a stale h or rho carried into the force, or a row
mismatch in the gather of the results fails this.
"""
import numpy as np
import pytest

import sph_inputs

KEYS = ("rho", "h", "nngb", "flags", "P", "c", "a", "dudt", "nngb_force")


@pytest.mark.parametrize("seed", [31, 32])
def test_sampled_step_equals_full_step(orc, seed):
    wl = sph_inputs.sod(n_lattice=32, seed=seed)
    wl.col("v")[:] = np.random.default_rng(seed).uniform(-0.3, 0.3, (wl.n, 3))
    full = orc.step(wl, with_kick_drift=False)
    rng = np.random.default_rng(seed + 100)
    x = wl.col("x")
    # random targets, plus the particles nearest the contact surfaces, where
    # the two halves' smoothing lengths differ by a factor of two
    near = np.argsort(np.minimum(np.abs(x[:, 0] - 0.5), np.minimum(x[:, 0], 1 - x[:, 0])))[:6]
    t = np.unique(np.concatenate([rng.choice(wl.n, 10, replace=False), near]))
    part = orc.step(wl, targets=t)
    for k in KEYS:
        assert np.array_equal(part[k], full[k][t]), k
    # the sample is a real subset: most particles were left out of the density
    mark = orc.ball_mark(x, wl.box, 2.0 * wl.h_cap, t)
    assert mark.sum() < 0.9 * wl.n


def test_sampled_step_single_target_at_the_wrap(orc):
    # one target on the periodic boundary: its ball wraps around the box
    wl = sph_inputs.sod(n_lattice=32, seed=33)
    x = wl.col("x")
    t = np.array([int(np.argmin(x[:, 0] + x[:, 1]))])
    full = orc.step(wl, with_kick_drift=False)
    part = orc.step(wl, targets=t)
    for k in KEYS:
        assert np.array_equal(part[k], full[k][t]), k
