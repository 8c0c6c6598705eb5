"""Pins of the oracle's level-hierarchy binning (per-particle h): Morton keys
against hand-derived codes and their inverse, the nesting of the levels
(a level-l cell is a key prefix), the level rule at its boundaries, and the
stable order by key."""
import math

import numpy as np
import pytest


def _centre(f, F):
    return (np.asarray(f, dtype=np.float64) + 0.5) / F


def test_morton_keys_of_hand_derived_cells(orc):
    F = 16
    cells = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (5, 3, 6), (15, 15, 15), (0, 0, 0)]
    # (5, 3, 6) = (101, 011, 110): bit 0 -> 0b011, bit 1 -> 0b110, bit 2 -> 0b101
    want = [1, 2, 4, 8, 3 + (6 << 3) + (5 << 6), 4095, 0]
    x = _centre(cells, F)
    key, lev, perm = orc.levels(x, np.full(len(cells), 1e-4), (1.0, 1.0, 1.0), 2, 4)
    assert key.tolist() == want


def _decode(key, bits):
    f = np.zeros((key.shape[0], 3), np.int64)
    k = key.astype(np.int64)
    for b in range(bits):
        for a in range(3):
            f[:, a] |= ((k >> (3 * b + a)) & 1) << b
    return f


def test_keys_invert_to_the_finest_cell_and_nest(orc):
    rng = np.random.default_rng(3)
    box = (1.0, 0.5, 2.0)
    x = rng.uniform(0.0, 1.0, (5000, 3)) * np.asarray(box)
    lmax = 9
    key, _, _ = orc.levels(x, np.full(5000, 1e-6), box, 2, lmax)
    F = 2 ** lmax
    # the inverse map gives floor(x F / L) on every axis
    assert np.array_equal(_decode(key, lmax), np.floor(x * (F / np.asarray(box))).astype(np.int64))
    # level l's cell is the key prefix: the keys of a hierarchy ending at l
    for l in (2, 5, 8):
        kl, _, _ = orc.levels(x, np.full(5000, 1e-6), box, 2, l)
        assert np.array_equal(key >> (3 * (lmax - l)), kl)


def test_level_rule_at_its_boundaries(orc):
    box = (1.0, 1.0, 0.5)                # caps follow the shortest edge
    lo, hi = 3, 7
    cap = {l: 0.5 * min(b / 2 ** l for b in box) for l in range(lo, hi + 1)}
    margin = 0.25
    h = [cap[5] / (1 + margin),                           # exactly at level 5's cap
         math.nextafter(cap[5] / (1 + margin), 1.0),      # just above it -> level 4
         cap[hi] / 4,                                     # small -> the finest level
         cap[lo] * 10,                                    # larger than every cap -> level_min
         float("nan"), float("inf"), 0.0, -1e-3]          # not finite and positive -> level_min
    want = [5, 4, hi, lo, lo, lo, lo, lo]
    # the exact-boundary case must hold in the product h (1 + margin)
    assert h[0] * (1 + margin) <= cap[5]
    assert h[1] * (1 + margin) > cap[5]
    x = np.full((len(h), 3), 0.1)
    _, lev, _ = orc.levels(x, np.asarray(h), box, lo, hi, margin)
    assert lev.tolist() == want


def test_order_is_stable_by_key(orc):
    rng = np.random.default_rng(4)
    x = rng.uniform(0.0, 1.0, (20000, 3))
    x[::7] = x[3]                        # many equal keys
    key, _, perm = orc.levels(x, np.full(20000, 1e-3), (1.0, 1.0, 1.0), 2, 6)
    assert np.array_equal(perm, np.argsort(key, kind="stable"))
    k = key[perm]
    assert np.all(np.diff(k) >= 0)
    same = np.flatnonzero(np.diff(k) == 0)
    assert np.all(perm[same + 1] > perm[same])


def test_bad_levels_are_refused(orc):
    x = np.zeros((1, 3))
    with pytest.raises(ValueError):
        orc.levels(x, np.ones(1), (1, 1, 1), 5, 4)


def test_positions_outside_the_box_clamp_into_the_edge_cells(orc):
    # as the cell binning: floor(x F / L) clamped to [0, F - 1]; NaN -> 0
    F = 2 ** 5
    x = np.array([[-0.3, 0.5, 0.5], [1.0, 0.5, 0.5], [2.7, 0.5, 0.5], [np.nan, 0.5, 0.5]])
    key, _, _ = orc.levels(x, np.full(4, 1e-3), (1.0, 1.0, 1.0), 2, 5)
    f = _decode(key, 5)
    assert f[:, 0].tolist() == [0, F - 1, F - 1, 0]
    assert np.all(f[:, 1] == F // 2) and np.all(f[:, 2] == F // 2)


def test_level_search_finds_every_force_pair_once(orc):
    # R24 by brute force on a small clustered set: with every h within its
    # level's cap, searching for each level l' the level-l' particles in the 27
    # cells of level min(l_i, l') around particle i finds every pair with
    # r < h_i + h_j exactly once (and the density's 27 cells of level l_i hold
    # every r < 2 h_i)
    rng = np.random.default_rng(11)
    n = 3000
    x = np.concatenate([rng.uniform(0, 1, (n // 3, 3)), 0.3 + 0.02 * rng.standard_normal((n - n // 3, 3))]) % 1.0
    lo, hi = 2, 6
    h = rng.uniform(0.004, 0.12, n)
    _, lev, _ = orc.levels(x, h, (1.0, 1.0, 1.0), lo, hi, 0.0)
    lev = lev.astype(int)
    cap = 0.5 * 2.0 ** -lev.astype(float)
    h = np.minimum(h, cap)                      # every h within its level's cap
    d = x[:, None, :] - x[None, :, :]
    d -= np.round(d)
    r = np.sqrt((d * d).sum(-1))
    for i in rng.choice(n, 200, replace=False):
        found = []
        for lp in range(lo, hi + 1):
            s = min(lev[i], lp)
            ci = np.floor(x[i] * 2 ** s).astype(int)
            cj = np.floor(x * 2 ** s).astype(int)
            dd = (cj - ci + 1) % 2 ** s            # neighbour cells -> 0, 1, 2
            near = np.all(dd <= 2, axis=1)
            found.extend(np.flatnonzero(near & (lev == lp)).tolist())
        assert len(found) == len(set(found))    # each candidate once
        pairs = set(np.flatnonzero((r[i] < h[i] + h) & (np.arange(n) != i)).tolist())
        assert pairs <= set(found), sorted(pairs - set(found))[:5]
        dens = set(np.flatnonzero(r[i] < 2 * h[i]).tolist())
        s = lev[i]
        cells = np.all((np.floor(x * 2 ** s).astype(int) - np.floor(x[i] * 2 ** s).astype(int) + 1) % 2 ** s <= 2,
                       axis=1)
        assert dens <= set(np.flatnonzero(cells).tolist())


def test_promotion_reproduces_the_single_cap_density(orc):
    # R23 on the oracle: Newton steps capped at each level's h_l, with every
    # particle that meets its cap moved one level up and recomputed from its
    # original h, end with exactly the h and density of the steps capped at
    # h_max alone (the same FP64 arithmetic on the same neighbours)
    rng = np.random.default_rng(13)
    n = 1500
    x = np.concatenate([rng.uniform(0, 1, (n // 2, 3)), 0.6 + 0.03 * rng.standard_normal((n - n // 2, 3))]) % 1.0
    m = np.full(n, 1.0 / n)
    eta = 0.5 * (3 * 48 / (4 * np.pi)) ** (1 / 3)
    lo, hi = 2, 6
    h0 = rng.uniform(0.01, 0.1, n)
    h_max = 0.5 * 2.0 ** -lo
    ref = orc.density(x, m, h0, (1.0, 1.0, 1.0), eta, h_max, 5, brute=True)
    _, lev, _ = orc.levels(x, h0, (1.0, 1.0, 1.0), lo, hi, 0.0)
    lev = lev.astype(int)
    rho = np.full(n, np.nan)
    hh = np.full(n, np.nan)
    todo = np.arange(n)
    promoted = 0
    for l in range(hi, lo - 1, -1):
        t = todo[lev[todo] == l]
        if t.size == 0:
            continue
        cap = min(h_max, 0.5 * 2.0 ** -l)
        o = orc.density(x, m, h0, (1.0, 1.0, 1.0), eta, cap, 5, brute=True, targets=t)
        up = (o["flags"] & orc.FLAG_HCAP) != 0 if l > lo else np.zeros(t.size, bool)
        rho[t[~up]] = o["rho"][~up]
        hh[t[~up]] = o["h"][~up]
        lev[t[up]] = l - 1
        promoted += int(up.sum())
    assert promoted > 0
    assert np.array_equal(rho, ref["rho"]) and np.array_equal(hh, ref["h"])
