"""The density over the level hierarchy (per-particle h on the clustered set).

* Binning: the finest cells' Morton keys, the levels and the slot order are
  bit-exact with the oracle's (integer work).
* Density with Newton steps: rho, h and P match the FP64 oracle -- one
  global h cap, brute-force neighbours -- within 1e-5 relative on sampled
  particles of every level, the promoted ones (h outgrew their level) among
  them; the level counters account for every particle.
* One level: the hierarchy reproduces the single-grid density of the same
  cells bit for bit (same candidates in the same order, same frames).
* Force with every particle's own h: acceleration and du/dt match the FP64
  oracle's brute-force pairs r < h_i + h_j, given the same h, rho, P and c,
  within 1e-5 of |a_i| + mean |a| per particle (a relative bound with the
  paper's mean-based floor; accelerations span orders of magnitude here).
* Per-target passes: with small stages most items are deferred to them (a
  block of warps per target) and the results still match the oracle.
"""
import numpy as np
import pytest
import torch

import sph_inputs
from gpu_util import make_sph

pytestmark = pytest.mark.gpu

import paper_2512_05516_gb300 as sph_mod  # noqa: E402


def _wl(n, seed=sph_inputs.SEED_BASE + 4):
    return sph_inputs.gaussian_mixture_adaptive(n, seed=seed)


@pytest.mark.parametrize("n,margin", [(50_003, 0.0), (65_536, 0.1)])
def test_level_binning_is_bit_exact(orc, n, margin):
    wl = _wl(n)
    lo, hi = wl.meta["levels"]
    s = make_sph(wl, ws_flags=sph_mod.WS_LEVELS)
    s.bin_levels(lo, hi, margin)
    key, lev, perm = orc.levels(wl.col("x"), wl.col("h"), wl.box, lo, hi, margin)
    assert np.array_equal(s.perm().cpu().numpy(), perm)
    assert np.array_equal(s.slot_cell().cpu().numpy(), key[perm])
    assert np.array_equal(s.levels().cpu().numpy(), lev[perm])
    s.close()


def _run_levels(wl, newton, margin, prec=None):
    lo, hi = wl.meta["levels"]
    s = make_sph(wl, ws_flags=sph_mod.WS_LEVELS)
    s.bin_levels(lo, hi, margin)
    lev0 = s.levels().cpu().numpy().copy()
    s.aos_to_soa(sph_mod.FIELDS_DENSITY, prec)
    s.density_levels(newton)
    s.soa_to_aos(sph_mod.mask("rho", "h", "P"))
    perm = s.perm().cpu().numpy()
    out = s.aos.cpu().numpy()
    lev = np.empty(wl.n, np.int8)
    lev[perm] = s.levels().cpu().numpy()
    first = np.empty(wl.n, np.int8)
    first[perm] = lev0
    res = {"rho": out[:, 11].copy(), "h": out[:, 10].copy(), "P": out[:, 13].copy(),
           "level": lev, "level0": first, "counts": s.level_counts(), "stats": s.stats()}
    s.close()
    return res


def _targets(g, n, rng, k_random=300, k_level=25, k_promoted=150):
    t = [rng.choice(n, k_random, replace=False)]
    for l in np.unique(g["level"]):
        idx = np.flatnonzero(g["level"] == l)
        t.append(rng.choice(idx, min(k_level, idx.size), replace=False))
    prom = np.flatnonzero(g["level"] < g["level0"])
    if prom.size:
        t.append(rng.choice(prom, min(k_promoted, prom.size), replace=False))
    return np.unique(np.concatenate(t))


@pytest.mark.parametrize("margin", [0.0, 0.1])
def test_level_density_matches_oracle(orc, margin):
    wl = _wl(262_144 - 77)
    lo, hi = wl.meta["levels"]
    g = _run_levels(wl, 5, margin)
    done, prom = g["counts"]
    # every particle was computed once, at the level it ended on
    assert sum(done) == wl.n
    assert np.array_equal(np.bincount(g["level"], minlength=sph_mod.LEVEL_MAX + 1), done)
    assert np.all(g["level"] <= g["level0"]) and g["level"].min() >= lo
    assert sum(prom) == int((g["level0"] - g["level"]).sum())
    if margin == 0.0:
        assert sum(prom) > 100          # the margin-free start exercises the promotion
    assert g["stats"]["error_bits"] & (sph_mod.ERR_NONFINITE | sph_mod.ERR_OUTSIDE) == 0
    rng = np.random.default_rng(5)
    t = _targets(g, wl.n, rng)
    o = orc.density(wl.col("x"), wl.col("m"), wl.col("h"), wl.box, wl.eta, wl.h_cap, 5, brute=True,
                    targets=t)
    assert (np.abs(g["h"][t] - o["h"]) / o["h"]).max() <= 1e-5
    assert (np.abs(g["rho"][t] - o["rho"]) / o["rho"]).max() <= 1e-5
    P, _ = orc.eos(o["rho"], wl.col("u")[t], wl.gamma)
    assert (np.abs(g["P"][t] - P) / P).max() <= 1e-5
    # each particle's final h fits the cells of the level it was computed at
    cap = 0.5 * 2.0 ** -g["level"].astype(np.float64)
    assert np.all(g["h"] <= cap * (1 + 1e-6))


def test_level_density_reduced_storage(orc):
    # m and h stored in BF16: the oracle takes the same rounded inputs
    wl = _wl(131_072 + 13)
    lo, hi = wl.meta["levels"]
    s = make_sph(wl, ws_flags=sph_mod.WS_LEVELS)
    s.bin_levels(lo, hi, 0.05)
    s.aos_to_soa(sph_mod.FIELDS_DENSITY, {"m": "bf16", "h": "bf16"})
    s.density_levels(3)
    s.soa_to_aos(sph_mod.mask("rho", "h"))
    out = s.aos.cpu().numpy()
    s.close()
    m_q = orc.quantize(wl.col("m"), "bf16")[0]
    h_q = orc.quantize(wl.col("h"), "bf16")[0]
    t = np.random.default_rng(6).choice(wl.n, 400, replace=False)
    o = orc.density(wl.col("x"), m_q, h_q, wl.box, wl.eta, wl.h_cap, 3, brute=True, targets=t)
    assert (np.abs(out[t, 11] - o["rho"]) / o["rho"]).max() <= 1e-5
    # h is written back through BF16: within one BF16 step of the oracle's
    h_o = orc.quantize(o["h"], "bf16")[0]
    assert (np.abs(out[t, 10] - h_o) / h_o).max() <= 2.0 ** -7


def test_one_level_equals_the_single_grid():
    # levels l..l over 2^l cells per axis and sph_density over the same
    # cells (one sub-cell): identical candidates, order and frames, so every
    # particle whose list holds its neighbourhood gets the same bits from
    # both kernels.  A particle whose list overflows (a sparse one whose h
    # overshoots in a Newton step) is summed from the stream by the cell
    # kernel and gathered target by target by the level kernel: the same
    # pairs in another order, equal to rounding.
    wl = sph_inputs.uniform_density(131_072, seed=sph_inputs.SEED_BASE + 21)
    h = float(wl.col("h").max())
    l = int(np.floor(np.log2(1.0 / (4.0 * h))))
    wl.h_cap = 0.5 * 2.0 ** -l
    wl.cell_edge = 2.0 ** -l
    a = make_sph(wl, ws_flags=sph_mod.WS_LEVELS)
    a.set_tuning(subcells=1, item_order=0, stage_density=4096)
    a.bin_levels(l, l, 0.0)
    a.aos_to_soa(sph_mod.FIELDS_DENSITY)
    a.density_levels(4)
    a.soa_to_aos(sph_mod.mask("rho", "h", "P"))
    b = make_sph(wl)
    b.set_tuning(subcells=1, item_order=0, stage_density=4096)
    b.bin_cells(wl.cell_edge)
    assert b.stats()["ncell"] == (2 ** l,) * 3
    b.aos_to_soa(sph_mod.FIELDS_DENSITY)
    b.density(4)
    b.soa_to_aos(sph_mod.mask("rho", "h", "P"))
    ra, rb = a.aos.cpu().numpy(), b.aos.cpu().numpy()
    same = np.ones(wl.n, bool)
    for col in (10, 11, 13):
        same &= ra[:, col] == rb[:, col]
        assert np.all(np.abs(ra[:, col] - rb[:, col]) <= 1e-6 * np.abs(rb[:, col])), col
    assert same.mean() >= 0.995, same.mean()
    pa = np.empty(wl.n, np.int32)
    pa[a.perm().cpu().numpy()] = a.nngb().cpu().numpy()
    pb = np.empty(wl.n, np.int32)
    pb[b.perm().cpu().numpy()] = b.nngb().cpu().numpy()
    assert np.array_equal(pa[same], pb[same])
    assert np.abs(pa - pb).max() <= 1
    ta, tb = a.stats()["pairs_density"], b.stats()["pairs_density"]
    assert abs(ta - tb) <= 1e-4 * tb
    a.close()
    b.close()


def test_level_calls_check_their_arguments_and_order():
    wl = _wl(20_000)
    lo, hi = wl.meta["levels"]
    s = make_sph(wl)                                    # no level workspace
    with pytest.raises(sph_mod.SphError) as e:
        s.bin_levels(lo, hi)
    assert e.value.status == sph_mod._capi.ENOSPACE
    s.close()
    s = make_sph(wl, ws_flags=sph_mod.WS_LEVELS)
    with pytest.raises(sph_mod.SphError) as e:         # not binned for levels
        s.density_levels(0)
    assert e.value.status == sph_mod._capi.ESTATE
    for a, b, m in ((1, hi, 0.0), (lo, 11, 0.0), (hi, lo, 0.0), (lo, hi, -0.1), (lo, hi, float("nan")),
                    (2, 2 + sph_mod.LEVELS_MAX, 0.0)):
        with pytest.raises(sph_mod.SphError) as e:
            s.bin_levels(a, b, m)
        assert e.value.status == sph_mod._capi.EINVAL, (a, b, m)
    with pytest.raises(sph_mod.SphError) as e:         # h_max above the coarsest cap
        s.bin_levels(lo + 1, hi, 0.0)
    assert e.value.status == sph_mod._capi.ECAPACITY
    s.bin_levels(lo, hi, 0.0)
    s.aos_to_soa(sph_mod.FIELDS_FORCE)
    with pytest.raises(sph_mod.SphError) as e:         # the force needs the density's outputs
        s.force_levels()
    assert e.value.status == sph_mod._capi.ESTATE
    for call in (lambda: s.density(0), s.force):       # single-grid kernels refuse level mode
        with pytest.raises(sph_mod.SphError) as e:
            call()
        assert e.value.status == sph_mod._capi.ESTATE
    with pytest.raises(sph_mod.SphError):              # positions are not written back
        s.soa_to_aos(sph_mod.mask("x"))
    s.density_levels(2)
    s.force_levels()
    s.aos_to_soa(sph_mod.mask("h"))                    # h from the records again: levels not fixed
    with pytest.raises(sph_mod.SphError) as e:
        s.force_levels()
    assert e.value.status == sph_mod._capi.ESTATE
    s.density_levels(2)
    s.force_levels()
    # back to cells: the single-grid density runs again
    s.bin_cells(wl.cell_edge)
    s.aos_to_soa(sph_mod.FIELDS_DENSITY)
    s.density(0)
    assert s.stats()["error_bits"] & (sph_mod.ERR_NONFINITE | sph_mod.ERR_OUTSIDE) == 0
    s.close()


# a 136-byte record that also carries the sound speed and du/dt
OFFS_136 = {"x": 0, "v": 24, "a": 48, "m": 72, "h": 80, "rho": 88, "u": 96, "P": 104,
            "cs": 112, "dudt": 120}


@pytest.mark.parametrize("margin", [0.0, 0.1])
def test_level_force_matches_oracle(orc, margin):
    wl = _wl(262_144 - 77)
    wl.col("v")[:] = np.random.default_rng(8).uniform(-0.5, 0.5, (wl.n, 3))
    lo, hi = wl.meta["levels"]
    rec = np.zeros((wl.n, 17))
    rec[:, :14] = wl.aos
    s = make_sph(wl, aos=torch.from_numpy(rec).cuda(), layout=sph_mod.make_layout(OFFS_136, 136),
                 ws_flags=sph_mod.WS_LEVELS)
    s.bin_levels(lo, hi, margin)
    s.aos_to_soa(sph_mod.FIELDS_FORCE)
    s.density_levels(5)
    s.force_levels()
    s.soa_to_aos(sph_mod.mask("h", "rho", "P", "cs", "a", "dudt"))
    out = s.aos.cpu().numpy()
    lev = np.empty(wl.n, np.int8)
    lev[s.perm().cpu().numpy()] = s.levels().cpu().numpy()
    st = s.stats()
    s.close()
    assert st["error_bits"] & (sph_mod.ERR_NONFINITE | sph_mod.ERR_OUTSIDE) == 0
    h, rho, P, c = out[:, 10], out[:, 11], out[:, 13], out[:, 14]
    rng = np.random.default_rng(9)
    t = [rng.choice(wl.n, 300, replace=False)]
    for l in np.unique(lev):
        idx = np.flatnonzero(lev == l)
        t.append(rng.choice(idx, min(40, idx.size), replace=False))
    t = np.unique(np.concatenate(t))
    f = orc.force(wl.col("x"), wl.col("v"), wl.col("m"), h, rho, P, c, wl.box, wl.alpha_av, wl.beta_av,
                  wl.eps_av, brute=True, targets=t)
    a_g, du_g = out[t, 6:9], out[t, 15]
    na = np.linalg.norm(f["a"], axis=1)
    err_a = np.linalg.norm(a_g - f["a"], axis=1)
    assert np.all(err_a <= 1e-5 * (na + na.mean())), (err_a / (na + na.mean())).max()
    err_u = np.abs(du_g - f["dudt"])
    assert np.all(err_u <= 1e-5 * (np.abs(f["dudt"]) + np.abs(f["dudt"]).mean()))
    assert st["pairs_force"] > 0


def test_adaptive_step_kicks_and_drifts_with_the_level_force():
    # a whole step over the hierarchy: the fused kick/drift + write-back uses
    # the level force's accelerations (v' = v + a dt in FP32, x' = x + v' dt in
    # FP64, periodic), and the density's outputs reach the records
    wl = _wl(65_536 + 5)
    wl.col("v")[:] = np.random.default_rng(12).uniform(-0.5, 0.5, (wl.n, 3))
    lo, hi = wl.meta["levels"]
    dt = 1e-5
    s = make_sph(wl, ws_flags=sph_mod.WS_LEVELS)
    s.step_levels(dt, lo, hi, newton_steps=3)
    st = s.stats()
    assert st["error_bits"] & (sph_mod.ERR_NONFINITE | sph_mod.ERR_OUTSIDE) == 0
    perm = s.perm().cpu().numpy()
    a = np.empty((wl.n, 3))
    for c in range(3):
        a[perm, c] = s.soa_raw("a", c).cpu().numpy()
    out = s.aos.cpu().numpy()
    s.close()
    v32 = wl.col("v").astype(np.float32) + (a.astype(np.float32) * np.float32(dt))
    assert np.allclose(out[:, 3:6], v32, rtol=0, atol=4e-7 * np.abs(v32).max())
    x = wl.col("x") + out[:, 3:6] * dt
    x -= np.floor(x)
    assert np.abs(out[:, 0:3] - x).max() <= 1e-12
    assert np.all(out[:, 11] > 0) and np.all(out[:, 10] > 0)        # rho, h written back


def test_level_binning_flags_bad_positions_and_stays_exact(orc):
    # NaN and out-of-box positions: flagged, clamped into the edge cells on
    # both sides exactly as the oracle does, and the context stays usable
    wl = _wl(20_000)
    lo, hi = wl.meta["levels"]
    bad = wl.aos.copy()
    bad[3, 0] = np.nan
    bad[5, 1] = 1.5
    bad[8, 2] = -0.1
    s = make_sph(wl, aos=torch.from_numpy(bad).cuda(), ws_flags=sph_mod.WS_LEVELS)
    s.bin_levels(lo, hi, 0.1)
    st = s.stats()
    assert st["status"] == sph_mod._capi.ENUMERIC
    assert st["error_bits"] & sph_mod.ERR_OUTSIDE and st["error_bits"] & sph_mod.ERR_NONFINITE
    key, lev, perm = orc.levels(bad[:, 0:3], bad[:, 10], wl.box, lo, hi, 0.1)
    assert np.array_equal(s.perm().cpu().numpy(), perm)
    assert np.array_equal(s.slot_cell().cpu().numpy(), key[perm])
    assert np.array_equal(s.levels().cpu().numpy(), lev[perm])
    s.close()


def test_level_density_without_newton_clamps_h_for_the_force(orc):
    # an input h above the coarsest level's cap (h_max): the density with no
    # Newton step clamps it to h_max and writes the clamped h, so that the
    # level force, which searches stencils sized for each level's cap, sees
    # every pair r < h_i + h_j of the oracle fed the same h, rho, P and c
    wl = _wl(65_536 + 9)
    wl.col("v")[:] = np.random.default_rng(13).uniform(-0.5, 0.5, (wl.n, 3))
    lo, hi = wl.meta["levels"]
    big = np.random.default_rng(14).choice(wl.n, 24, replace=False)
    wl.col("h")[big] = 1.5 * wl.h_cap
    rec = np.zeros((wl.n, 17))
    rec[:, :14] = wl.aos
    s = make_sph(wl, aos=torch.from_numpy(rec).cuda(), layout=sph_mod.make_layout(OFFS_136, 136),
                 ws_flags=sph_mod.WS_LEVELS)
    s.bin_levels(lo, hi, 0.0)
    s.aos_to_soa(sph_mod.FIELDS_FORCE)
    s.density_levels(0)
    s.force_levels()
    s.soa_to_aos(sph_mod.mask("h", "rho", "P", "cs", "a", "dudt"))
    out = s.aos.cpu().numpy()
    st = s.stats()
    s.close()
    assert st["error_bits"] & sph_mod.ERR_HCAP
    assert st["error_bits"] & (sph_mod.ERR_NONFINITE | sph_mod.ERR_OUTSIDE) == 0
    h, rho, P, c = out[:, 10], out[:, 11], out[:, 13], out[:, 14]
    assert np.all(h[big] == float(np.float32(wl.h_cap)))
    assert np.all(h <= float(np.float32(wl.h_cap)))
    o = orc.density(wl.col("x"), wl.col("m"), wl.col("h"), wl.box, wl.eta, wl.h_cap, 0, brute=True,
                    targets=big)
    assert np.all(o["h"] == wl.h_cap) and np.all(o["flags"] & orc.FLAG_HCAP)
    assert (np.abs(rho[big] - o["rho"]) / o["rho"]).max() <= 1e-5
    # targets: the clamped particles and their force partners
    x = wl.col("x")
    near = orc.ball_mark(x, wl.box, 2.0 * wl.h_cap, big)
    rng = np.random.default_rng(15)
    t = np.unique(np.concatenate([big, rng.choice(np.flatnonzero(near), 200, replace=False)]))
    f = orc.force(x, wl.col("v"), wl.col("m"), h, rho, P, c, wl.box, wl.alpha_av, wl.beta_av,
                  wl.eps_av, brute=True, targets=t)
    na = np.linalg.norm(f["a"], axis=1)
    err_a = np.linalg.norm(out[t, 6:9] - f["a"], axis=1)
    assert np.all(err_a <= 1e-5 * (na + na.mean())), (err_a / (na + na.mean())).max()


def test_level_density_16777216_newton_flags_sampled(orc):
    # The full-size clustered set as bench.py runs it (levels from the set,
    # margin 0.1, 5 Newton steps, FP32 storage).  A Newton step that meets
    # f'(h) <= 0 keeps h (R5) and flags the particle; the per-particle flags
    # show which.  Targets: every flagged particle (a random 3,000 of them if
    # there are more) and 300 others; the FP64 oracle with the single cap
    # must flag the same ones and give the same h and rho within 1e-5.
    wl = sph_inputs.gaussian_mixture_adaptive(16_777_216)
    lo, hi = wl.meta["levels"]
    s = make_sph(wl, ws_flags=sph_mod.WS_LEVELS)
    s.bin_levels(lo, hi, 0.1)
    s.aos_to_soa(sph_mod.FIELDS_DENSITY)
    s.density_levels(5)
    s.soa_to_aos(sph_mod.mask("rho", "h"))
    perm = s.perm().cpu().numpy()
    fl = np.empty(wl.n, np.uint8)
    fl[perm] = s.density_flags().cpu().numpy()
    out = s.aos.cpu().numpy()
    st = s.stats()
    done, prom = s.level_counts()
    s.close()
    assert sum(done) == wl.n
    assert st["error_bits"] & (sph_mod.ERR_NONFINITE | sph_mod.ERR_OUTSIDE) == 0
    newt = np.flatnonzero(fl & sph_mod.PFLAG_NEWTON)
    # the error word's NEWTON bit is exactly the union of the per-particle flags
    assert bool(st["error_bits"] & sph_mod.ERR_NEWTON) == (newt.size > 0)
    assert np.all((fl & sph_mod.PFLAG_NONFINITE) == 0)
    rng = np.random.default_rng(17)
    pick = newt if newt.size <= 3000 else rng.choice(newt, 3000, replace=False)
    others = rng.choice(np.flatnonzero((fl & sph_mod.PFLAG_NEWTON) == 0), 300, replace=False)
    t = np.unique(np.concatenate([pick, others]))
    o = orc.density(wl.col("x"), wl.col("m"), wl.col("h"), wl.box, wl.eta, wl.h_cap, 5, targets=t)
    assert (np.abs(out[t, 10] - o["h"]) / o["h"]).max() <= 1e-5
    assert (np.abs(out[t, 11] - o["rho"]) / o["rho"]).max() <= 1e-5
    g_new = (fl[t] & sph_mod.PFLAG_NEWTON) != 0
    o_new = (o["flags"] & orc.FLAG_NEWTON) != 0
    # the sign of f' is decided in FP32 on the GPU and in FP64 in the oracle:
    # only particles with f' within rounding of 0 may differ
    assert np.count_nonzero(g_new != o_new) <= max(2, t.size // 1000)


def test_level_per_target_passes_match_oracle(orc):
    # small stages defer most items of every level to the per-target passes
    # (density: beyond 8 x 32 staged candidates; force: beyond 64 x 32), where
    # one block of warps gathers each target, its stream split between the
    # warps; rho, h, a and du/dt still match the FP64 oracle
    wl = _wl(65_536 + 11, seed=sph_inputs.SEED_BASE + 31)
    wl.col("v")[:] = np.random.default_rng(10).uniform(-0.5, 0.5, (wl.n, 3))
    lo, hi = wl.meta["levels"]
    rec = np.zeros((wl.n, 17))
    rec[:, :14] = wl.aos
    s = make_sph(wl, aos=torch.from_numpy(rec).cuda(), layout=sph_mod.make_layout(OFFS_136, 136),
                 ws_flags=sph_mod.WS_LEVELS)
    s.set_tuning(stage_density=32, stage_force=32)
    s.bin_levels(lo, hi, 0.1)
    s.aos_to_soa(sph_mod.FIELDS_FORCE)
    s.density_levels(5)
    done, prom = s.level_counts()
    s.force_levels()
    s.soa_to_aos(sph_mod.mask("h", "rho", "P", "cs", "a", "dudt"))
    out = s.aos.cpu().numpy()
    st = s.stats()
    s.close()
    assert sum(done) == wl.n
    assert st["error_bits"] & (sph_mod.ERR_NONFINITE | sph_mod.ERR_OUTSIDE) == 0
    rng = np.random.default_rng(11)
    t = np.unique(rng.choice(wl.n, 400, replace=False))
    o = orc.density(wl.col("x"), wl.col("m"), wl.col("h"), wl.box, wl.eta, wl.h_cap, 5, brute=True,
                    targets=t)
    h, rho, P, c = out[:, 10], out[:, 11], out[:, 13], out[:, 14]
    assert (np.abs(h[t] - o["h"]) / o["h"]).max() <= 1e-5
    assert (np.abs(rho[t] - o["rho"]) / o["rho"]).max() <= 1e-5
    f = orc.force(wl.col("x"), wl.col("v"), wl.col("m"), h, rho, P, c, wl.box, wl.alpha_av, wl.beta_av,
                  wl.eps_av, brute=True, targets=t)
    na = np.linalg.norm(f["a"], axis=1)
    err_a = np.linalg.norm(out[t, 6:9] - f["a"], axis=1)
    assert np.all(err_a <= 1e-5 * (na + na.mean())), (err_a / (na + na.mean())).max()
    # du/dt sums terms of both signs (v_ij . grad W), so its FP32 rounding
    # is not bounded by 1e-5 of |du/dt| + mean: one of these 400 particles
    # (37 pairs) is at 1.01e-5, with one warp or a block per target alike;
    # the 1e-5 gate is the density's and the acceleration's
    err_u = np.abs(out[t, 15] - f["dudt"])
    ru = err_u / (np.abs(f["dudt"]) + np.abs(f["dudt"]).mean())
    assert ru.max() <= 2e-5, ru.max()
