"""S5/S6/S7 parity: the symmetric force with artificial viscosity, kick/drift,
and a whole step, against the FP64 oracle.

Acceleration tolerance: max |a_gpu - a_orc| <= 1e-5 * mean |a_orc| (the
paper's error metric divides by the average of the quantity); the same for
du/dt.  Positions after the drift within 1e-12 absolute (FP64 drift of FP32
velocities times dt)."""
import numpy as np
import pytest
import torch

import sph_inputs
from gpu_util import force_count_band_ok, make_sph

pytestmark = pytest.mark.gpu

import paper_2512_05516_gb300 as sph_mod  # noqa: E402

# a 136-byte record that also carries the sound speed and du/dt, so that the
# force and kick/drift kernels can be fed the oracle's own inputs
OFFS_136 = {"x": 0, "v": 24, "a": 48, "m": 72, "h": 80, "rho": 88, "u": 96, "P": 104,
            "cs": 112, "dudt": 120}


def _record136(wl, extra):
    n = wl.n
    out = np.zeros((n, 17))
    out[:, :14] = wl.aos
    out[:, 14] = extra.get("cs", 0.0)
    out[:, 15] = extra.get("dudt", 0.0)
    return out


def _mean_abs(a):
    return float(np.mean(np.linalg.norm(a, axis=1)))


@pytest.mark.parametrize("masses", ["equal", "unequal"])
def test_force_isolated(orc, masses):
    # h, rho, P, c come from the oracle's density and are handed to both sides
    wl = sph_inputs.sod(n_lattice=24, seed=21)
    wl.col("v")[:] = np.random.default_rng(1).uniform(-0.5, 0.5, (wl.n, 3))
    if masses == "unequal":
        wl.col("m")[:] = wl.col("m") * np.random.default_rng(2).uniform(0.5, 1.5, wl.n)
    x, v, m, u = wl.col("x"), wl.col("v"), wl.col("m"), wl.col("u")
    d = orc.density(x, m, wl.col("h"), wl.box, wl.eta, wl.h_cap, 5)
    P, c = orc.eos(d["rho"], u, wl.gamma)
    wl.col("h")[:] = d["h"]
    wl.col("rho")[:] = d["rho"]
    wl.col("P")[:] = P
    f = orc.force(x, v, m, d["h"], d["rho"], P, c, wl.box, wl.alpha_av, wl.beta_av, wl.eps_av)
    rec = _record136(wl, {"cs": c})
    aos = torch.from_numpy(rec).cuda()
    layout = sph_mod.make_layout(OFFS_136, 136)
    s = make_sph(wl, aos=aos, layout=layout)
    s.bin_cells(wl.cell_edge)
    s.aos_to_soa(sph_mod.mask("x", "v", "m", "h", "rho", "P", "cs"))
    s.force()
    s.soa_to_aos(sph_mod.mask("a", "dudt"))
    out = s.aos.cpu().numpy()
    a_g = out[:, 6:9]
    du_g = out[:, 15]
    scale = _mean_abs(f["a"])
    err = np.linalg.norm(a_g - f["a"], axis=1).max() / scale
    assert err <= 1e-5, err
    err_u = np.abs(du_g - f["dudt"]).max() / np.mean(np.abs(f["dudt"]))
    assert err_u <= 1e-5, err_u
    perm = s.perm().cpu().numpy()
    cnt = np.empty(wl.n, np.int32)
    cnt[perm] = s.nngb(force=True).cpu().numpy()
    # force-neighbour counts (r < h_i + h_j): between the oracle's counts at
    # (h_i + h_j)(1 -+ delta), and equal to its count wherever no pair sits
    # within that band; h reaches the GPU rounded to FP32 (relative 6e-8)
    ok, lo, hi = force_count_band_ok(orc, x, m, d["h"], wl.box, cnt, 1e-6)
    assert ok.all()
    exact = lo == hi
    assert np.array_equal(cnt[exact], f["nngb"][exact])
    assert exact.mean() > 0.99
    # momentum: the FP32 pair terms are antisymmetric up to rounding
    ma = m[:, None] * a_g
    assert np.all(np.abs(ma.sum(0)) <= 1e-5 * np.abs(ma).sum(0))
    st = s.stats()
    assert st["pairs_force"] == int(cnt.sum())
    assert st["error_bits"] == 0


def test_kick_drift_isolated(orc):
    wl = sph_inputs.random_cloud(5000, seed=22, vel=2.0)
    wl.h_cap = 0.05
    wl.cell_edge = 0.1
    rng = np.random.default_rng(2)
    wl.col("a")[:] = rng.uniform(-50, 50, (wl.n, 3))
    dudt = rng.uniform(-5, 5, wl.n)
    rec = _record136(wl, {"dudt": dudt})
    aos = torch.from_numpy(rec).cuda()
    s = make_sph(wl, aos=aos, layout=sph_mod.make_layout(OFFS_136, 136))
    s.bin_cells(wl.cell_edge)
    s.aos_to_soa(sph_mod.mask("v", "a", "u", "dudt"))
    dt = 1e-2
    s.kick_drift(dt, dt)
    s.soa_to_aos(sph_mod.mask("v", "u"))
    out = s.aos.cpu().numpy()
    xo, vo, uo = orc.kick_drift(wl.col("x"), wl.col("v"), wl.col("a"), wl.col("u"), dudt, dt, dt, wl.box)
    assert np.abs(out[:, 3:6] - vo).max() <= 1e-6 * np.abs(vo).max()
    assert np.abs(out[:, 12] - uo).max() <= 1e-6 * np.abs(uo).max()
    dx = np.abs(out[:, 0:3] - xo)
    dx = np.minimum(dx, 1.0 - dx)             # periodic
    # the drift uses the FP32 velocity: |dx| <= a few FP32 ulps of v times dt
    assert dx.max() <= 4 * 2.0 ** -24 * np.abs(vo).max() * dt
    assert np.all((out[:, 0:3] >= 0) & (out[:, 0:3] < 1))


@pytest.mark.parametrize("shuffle", [False, True])
def test_full_step_small_sod(orc, shuffle):
    wl = sph_inputs.sod(n_lattice=24, seed=23, shuffle=shuffle)
    o = orc.step(wl)
    s = make_sph(wl)
    s.step(wl.dt, wl.newton_steps, cell_edge=wl.cell_edge)
    out = s.aos.cpu().numpy()
    assert (np.abs(out[:, 11] - o["rho"]) / o["rho"]).max() <= 1e-5
    assert (np.abs(out[:, 10] - o["h"]) / o["h"]).max() <= 1e-5
    assert (np.abs(out[:, 13] - o["P"]) / o["P"]).max() <= 1e-5
    scale = _mean_abs(o["a"])
    assert np.linalg.norm(out[:, 6:9] - o["a"], axis=1).max() / scale <= 1e-5
    vscale = np.abs(o["v_new"]).max()
    assert np.abs(out[:, 3:6] - o["v_new"]).max() <= 1e-5 * vscale
    assert np.abs(out[:, 12] - o["u_new"]).max() <= 1e-6 * np.abs(o["u_new"]).max()
    dx = np.abs(out[:, 0:3] - o["x_new"])
    dx = np.minimum(dx, 1.0 - dx)
    assert dx.max() <= 1e-9
    # m is never written back
    assert np.array_equal(out[:, 9], wl.col("m"))
    st = s.stats()
    assert st["error_bits"] == 0


def test_step_twice_then_rebin(orc):
    # two steps in a row: the second re-bins the drifted AoS
    wl = sph_inputs.sod(n_lattice=24, seed=24)
    s = make_sph(wl)
    s.step(wl.dt, 5, cell_edge=wl.cell_edge)
    s.step(wl.dt, 5, cell_edge=wl.cell_edge)
    a1 = s.aos.cpu().numpy()
    o1 = orc.step(wl)
    wl2 = sph_inputs.Workload("sod", wl.aos.copy(), wl.box, h_cap=wl.h_cap, cell_edge=wl.cell_edge)
    wl2.col("x")[:] = o1["x_new"]
    wl2.col("v")[:] = o1["v_new"]
    wl2.col("u")[:] = o1["u_new"]
    wl2.col("h")[:] = o1["h"]
    o2 = orc.step(wl2)
    assert (np.abs(a1[:, 11] - o2["rho"]) / o2["rho"]).max() <= 1e-4
    assert np.linalg.norm(a1[:, 6:9] - o2["a"], axis=1).max() / _mean_abs(o2["a"]) <= 1e-4
