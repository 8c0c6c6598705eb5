"""Parity at the benchmark sizes, in the launch configuration bench.py times:
the CUDA step runs on every particle, the FP64 oracle evaluates a sample of
particles one by one (every particle its sample needs included), and the
two are compared on that sample.  Invariants that hold at any size (momentum
balance, neighbour-count bounds, positions inside the box) are checked on
every particle."""
import math

import numpy as np
import pytest
import torch

import sph_inputs
from gpu_util import count_band_ok, force_count_band_ok, make_sph

pytestmark = pytest.mark.gpu


def _sample(wl, n_rand, extra=(), seed=0):
    rng = np.random.default_rng(seed)
    t = set(rng.choice(wl.n, n_rand, replace=False).tolist())
    t.update(int(i) for i in extra)
    return np.array(sorted(t), dtype=np.int64)


def _check_step(orc, wl, out, targets, prec=None):
    o = orc.step(wl, targets=targets)
    rho, h, a = out[targets, 11], out[targets, 10], out[targets, 6:9]
    assert (np.abs(rho - o["rho"]) / o["rho"]).max() <= 1e-5
    assert (np.abs(h - o["h"]) / o["h"]).max() <= 1e-5
    scale = np.mean(np.linalg.norm(o["a"], axis=1))
    assert np.linalg.norm(a - o["a"], axis=1).max() / scale <= 1e-5
    return o


def test_sod_1072476_sampled(orc):
    wl = sph_inputs.sod()
    assert wl.n == 1_072_476
    x = wl.col("x")
    # random particles plus those nearest the two contact surfaces (x = 0.5, x = 0)
    near = np.argsort(np.minimum(np.abs(x[:, 0] - 0.5), np.minimum(x[:, 0], 1 - x[:, 0])))[:150]
    targets = _sample(wl, 250, near, seed=1)
    s = make_sph(wl)                     # default launch shapes, as bench.py
    s.step(wl.dt, wl.newton_steps, cell_edge=wl.cell_edge)
    out = s.aos.cpu().numpy()
    st = s.stats()
    assert st["error_bits"] == 0
    o = _check_step(orc, wl, out, targets)
    # every particle: the force balance and the box
    m = wl.col("m")
    ma = m[:, None] * out[:, 6:9]
    assert np.all(np.abs(ma.sum(0)) <= 1e-5 * np.abs(ma).sum(0))
    assert np.all((out[:, 0:3] >= 0) & (out[:, 0:3] < 1))
    # neighbour counts of the final density pass: the sample's match the
    # oracle's up to pairs at the edge of the support; all particles sit near
    # the ~48 the smoothing-length iteration aims for (the jittered lattice
    # and the contact spread it)
    perm = s.perm().cpu().numpy()
    cnt = np.empty(wl.n, np.int32)
    cnt[perm] = s.nngb().cpu().numpy()
    # the sample's density counts: within the band of the oracle's counts at
    # h (1 -+ 2e-5) around the oracle's own h (h itself is held to 1e-5)
    h_ref = o["h_all"].copy()
    ok, lo, hi = count_band_ok(orc, wl, h_ref, cnt[targets], 2e-5, targets=targets)
    assert ok.all()
    assert np.array_equal(cnt[targets][lo == hi], o["nngb"][lo == hi])
    assert 12 <= cnt.min() and cnt.max() <= 120
    # the sample's force counts (r < h_i + h_j) by the same band rule, on
    # the h the oracle's sampled force read
    cntf = np.empty(wl.n, np.int32)
    cntf[perm] = s.nngb(force=True).cpu().numpy()
    ok, lo, hi = force_count_band_ok(orc, x, m, h_ref, wl.box, cntf[targets], 2e-5,
                                     targets=targets)
    assert ok.all()
    assert np.array_equal(cntf[targets][lo == hi], o["nngb_force"][lo == hi])


def test_long_run_33554432_sampled(orc):
    wl = sph_inputs.long_run()
    assert wl.n == 33_554_432
    targets = _sample(wl, 200, seed=2)
    s = make_sph(wl, ws_flags=1)
    s.bin_cells(wl.cell_edge, reorder=True)      # cell-ordered records, as bench.py
    import paper_2512_05516_gb300 as sph
    s.aos_to_soa(sph.FIELDS_FORCE)
    s.density(0)
    s.force()
    s.soa_to_aos(sph.mask("rho", "a", "P"))
    out = s.aos.cpu().numpy()
    st = s.stats()
    assert st["error_bits"] == 0
    # the AoS was reordered: find each sampled particle by its (unchanged) position
    perm = np.lexsort((wl.col("x")[:, 2], wl.col("x")[:, 1], wl.col("x")[:, 0]))
    perm_out = np.lexsort((out[:, 2], out[:, 1], out[:, 0]))
    where = np.empty(wl.n, np.int64)
    where[perm] = perm_out
    d = orc.density(wl.col("x"), wl.col("m"), wl.col("h"), wl.box, wl.eta, wl.h_cap, 0,
                    targets=targets)
    rho = out[where[targets], 11]
    assert (np.abs(rho - d["rho"]) / d["rho"]).max() <= 1e-5
    del out


def test_gaussian_mixture_uneven_cells(orc):
    # the uneven-occupancy workload at 1/64 of its size: the same 8 Gaussians
    # and background with the same global-h rule, so the densest cell holds
    # ~17,000 particles (mean ~12) and a core particle ~26,000 neighbours,
    # which stream through the stage in chunks
    wl = sph_inputs.gaussian_mixture(n=1 << 18)
    s = make_sph(wl)
    import paper_2512_05516_gb300 as sph
    s.bin_cells(wl.cell_edge)
    st = s.stats()
    assert st["max_occupancy"] > 10000
    s.aos_to_soa(sph.FIELDS_DENSITY)
    s.density(0)
    s.soa_to_aos(sph.mask("rho"))
    rho = s.aos.cpu().numpy()[:, 11]
    x = wl.col("x")
    centre = wl.meta["centres"][0]                 # the sigma = 0.01 Gaussian
    d = x - centre
    d -= np.round(d)
    core = np.argsort(np.sum(d * d, axis=1))[:40]
    targets = _sample(wl, 160, core, seed=3)
    o = orc.density(x, wl.col("m"), wl.col("h"), wl.box, wl.eta, wl.h_cap, 0, targets=targets)
    assert (np.abs(rho[targets] - o["rho"]) / o["rho"]).max() <= 1e-5
    assert o["nngb"].max() > 20000                  # some targets sit in the dense core
    cnt = np.empty(wl.n, np.int32)
    cnt[s.perm().cpu().numpy()] = s.nngb().cpu().numpy()
    ok, lo, hi = count_band_ok(orc, wl, wl.col("h"), cnt[targets], 4e-6, targets=targets)
    assert ok.all()
    assert np.array_equal(cnt[targets][lo == hi], o["nngb"][lo == hi])


def test_gaussian_mixture_16777216_bf16_sampled(orc):
    # the uneven-occupancy workload at full size, BF16 storage of v, m, h, u
    # as bench.py runs it: densest cell ~65,000 particles, core particles with
    # ~10^5 neighbours; the oracle evaluates sampled targets (core ones
    # included) on the same BF16-rounded m and h (mode Q)
    import paper_2512_05516_gb300 as sph
    wl = sph_inputs.gaussian_mixture(n=16_777_216)
    assert wl.n == 16_777_216
    prec = {"v": "bf16", "m": "bf16", "h": "bf16", "u": "bf16"}
    s = make_sph(wl)
    s.bin_cells(wl.cell_edge)
    st = s.stats()
    assert st["max_occupancy"] > 60000
    s.aos_to_soa(sph.FIELDS_DENSITY, prec)
    s.density(0)
    s.soa_to_aos(sph.mask("rho"))
    rho = s.aos.cpu().numpy()[:, 11]
    assert s.stats()["error_bits"] == 0
    x = wl.col("x")
    centre = wl.meta["centres"][0]                 # the sigma = 0.01 Gaussian
    d = x - centre
    d -= np.round(d)
    core = np.argsort(np.sum(d * d, axis=1))[:40]
    targets = _sample(wl, 160, core, seed=4)
    mq = orc.quantize(wl.col("m"), "bf16")[0]
    hq = orc.quantize(wl.col("h"), "bf16")[0]
    o = orc.density(x, mq, hq, wl.box, wl.eta, wl.h_cap, 0, targets=targets)
    assert (np.abs(rho[targets] - o["rho"]) / o["rho"]).max() <= 1e-5
    assert o["nngb"].max() > 50000                  # some targets sit in the dense core
    cnt = np.empty(wl.n, np.int32)
    cnt[s.perm().cpu().numpy()] = s.nngb().cpu().numpy()
    ok, lo, hi = count_band_ok(orc, wl, hq, cnt[targets], 4e-6, targets=targets, m=mq)
    assert ok.all()
    assert np.array_equal(cnt[targets][lo == hi], o["nngb"][lo == hi])
    s.close()
