"""Reduced-precision storage (Table 2 formats and bfloat16) in the pair
kernels.  Storage only: the kernels decode to FP32 and compute in FP32, so
against the FP64 oracle fed the *same quantised inputs* (mode Q) they must
agree to the FP32 tolerance; against the unquantised FP64 oracle (mode T) the
storage error is reported and bounded loosely."""
import numpy as np
import pytest
import torch

import sph_inputs
from gpu_util import make_sph

pytestmark = pytest.mark.gpu

import paper_2512_05516_gb300 as sph_mod  # noqa: E402

FMTS = ["bf16", "fp16", "m16", "m10"]
OFFS_136 = {"x": 0, "v": 24, "a": 48, "m": 72, "h": 80, "rho": 88, "u": 96, "P": 104,
            "cs": 112, "dudt": 120}


def _q(orc, vals, fmt):
    return orc.quantize(np.asarray(vals).ravel(), fmt)[0].reshape(np.shape(vals))


@pytest.mark.parametrize("pos", ["fp32", "fp16"])
@pytest.mark.parametrize("fmt", FMTS)
def test_density_fixed_h_mode_q(orc, fmt, pos):
    wl = sph_inputs.uniform_density()
    # room above h for values that round up in the storage format (7 cells stay)
    wl.h_cap = 1.01 * wl.meta["h"]
    s = make_sph(wl)
    s.bin_cells(wl.cell_edge)
    assert tuple(s.nc) == (7, 7, 7)
    s.aos_to_soa(sph_mod.mask("x", "m", "h"), {"x": pos, "m": fmt, "h": fmt})
    s.density(0)
    s.soa_to_aos(sph_mod.mask("rho"))
    rho = s.aos.cpu().numpy()[:, 11]
    xq, _ = orc.cell_relative(wl.col("x"), wl.box, s.nc, pos)
    mq, hq = _q(orc, wl.col("m"), fmt), _q(orc, wl.col("h"), fmt)
    o = orc.density(xq, mq, hq, wl.box, wl.eta, wl.h_cap, 0)
    assert (np.abs(rho - o["rho"]) / o["rho"]).max() <= 1e-5
    # against the unquantised FP64 density: the storage error alone
    t = orc.density(wl.col("x"), wl.col("m"), wl.col("h"), wl.box, wl.eta, wl.h_cap, 0)
    err_t = np.sqrt(np.mean((rho - t["rho"]) ** 2)) / np.mean(t["rho"])
    bound = {"bf16": 2e-2, "fp16": 4e-3, "m16": 2e-4, "m10": 1e-2}[fmt]
    if pos == "fp16":
        bound = max(bound, 4e-3)
    assert err_t <= bound, err_t


@pytest.mark.parametrize("fmt", FMTS)
def test_force_mode_q(orc, fmt):
    wl = sph_inputs.sod(n_lattice=24, seed=41)
    rng = np.random.default_rng(4)
    wl.col("v")[:] = rng.uniform(-0.5, 0.5, (wl.n, 3))
    x, m, u = wl.col("x"), wl.col("m"), wl.col("u")
    d = orc.density(x, m, wl.col("h"), wl.box, wl.eta, wl.h_cap, 5)
    P, c = orc.eos(d["rho"], u, wl.gamma)
    wl.col("h")[:] = d["h"]
    wl.col("rho")[:] = d["rho"]
    wl.col("P")[:] = P
    rec = np.zeros((wl.n, 17))
    rec[:, :14] = wl.aos
    rec[:, 14] = c
    s = make_sph(wl, aos=torch.from_numpy(rec).cuda(), layout=sph_mod.make_layout(OFFS_136, 136))
    s.bin_cells(wl.cell_edge)
    s.aos_to_soa(sph_mod.mask("x", "v", "m", "h", "rho", "P", "cs"), {"v": fmt, "m": fmt, "h": fmt})
    s.force()
    s.soa_to_aos(sph_mod.mask("a", "dudt"))
    out = s.aos.cpu().numpy()
    vq, mq, hq = _q(orc, wl.col("v"), fmt), _q(orc, m, fmt), _q(orc, d["h"], fmt)
    f = orc.force(x, vq, mq, hq, d["rho"], P, c, wl.box, wl.alpha_av, wl.beta_av, wl.eps_av)
    scale = np.mean(np.linalg.norm(f["a"], axis=1))
    err = np.linalg.norm(out[:, 6:9] - f["a"], axis=1).max() / scale
    assert err <= 1e-5, err
    err_u = np.abs(out[:, 15] - f["dudt"]).max() / np.mean(np.abs(f["dudt"]))
    assert err_u <= 1e-5, err_u


@pytest.mark.parametrize("fmt", FMTS)
def test_newton_h_and_kick_drift_store_in_format(orc, fmt):
    # density with Newton writes h in the storage format; kick/drift writes v, u
    wl = sph_inputs.sod(n_lattice=24, seed=42)
    s = make_sph(wl)
    prec = {"v": fmt, "m": fmt, "h": fmt, "u": fmt}
    s.step(wl.dt, 5, prec=prec, cell_edge=wl.cell_edge)
    out = s.aos.cpu().numpy()
    perm = s.perm().cpu().numpy()
    # every stored value is exactly representable in the format
    for col in (10, 3, 4, 5, 12):      # h, v, u
        vals = out[:, col]
        assert np.array_equal(_q(orc, vals, fmt), vals), col
    # mode Q density/h: the oracle on the quantised inputs, its h rounded to
    # the format; they agree within one unit of the format
    xq = wl.col("x")
    mq, hq, uq = _q(orc, wl.col("m"), fmt), _q(orc, wl.col("h"), fmt), _q(orc, wl.col("u"), fmt)
    xq, _ = orc.cell_relative(xq, wl.box, s.nc, "fp32")
    o = orc.density(xq, mq, hq, wl.box, wl.eta, wl.h_cap, 5)
    ulp = {"bf16": 2.0 ** -7, "fp16": 2.0 ** -10, "m16": 2.0 ** -16, "m10": 2.0 ** -10}[fmt]
    assert (np.abs(out[:, 10] - o["h"]) / o["h"]).max() <= 1.01 * ulp + 1e-5
    assert (np.abs(out[:, 11] - o["rho"]) / o["rho"]).max() <= 1e-5


def test_fp16_positions_relative_to_cell(orc):
    # positions stored as FP16 offsets from the cell origin keep ~11 bits of
    # the cell edge; the density error against FP64 follows from that
    wl = sph_inputs.sod(n_lattice=24, seed=43)
    s = make_sph(wl)
    s.bin_cells(wl.cell_edge)
    s.aos_to_soa(sph_mod.FIELDS_DENSITY, {"x": "fp16"})
    s.density(5)
    s.soa_to_aos(sph_mod.mask("rho", "h"))
    out = s.aos.cpu().numpy()
    xq, _ = orc.cell_relative(wl.col("x"), wl.box, s.nc, "fp16")
    o = orc.density(xq, wl.col("m"), wl.col("h"), wl.box, wl.eta, wl.h_cap, 5)
    assert (np.abs(out[:, 11] - o["rho"]) / o["rho"]).max() <= 1e-5


def test_fp16_storage_scale_on_a_subnormal_mass(orc):
    # lattice 48: m = 1/48^3 = 9.0e-6, an FP16 subnormal.  Unscaled, the
    # stored mass loses ~0.3 %; with the power-of-two storage scale the
    # codes are the oracle's codes of m 2^e, the density matches the
    # oracle on those inputs (mode Q) to FP32 accuracy, and against FP64
    # (mode T) it stays within 1e-3.
    wl = sph_inputs.sod(n_lattice=48, seed=44)
    m, h = wl.col("m"), wl.col("h")
    e = sph_mod.suggest_scale(float(m.max()), "fp16")
    assert e > 0
    s = make_sph(wl)
    s.bin_cells(wl.cell_edge)
    t = orc.density(wl.col("x"), m, h, wl.box, wl.eta, wl.h_cap, 5)
    res = {}
    for scaled in (False, True):
        s.set_scale({"m": e if scaled else 0})
        assert s.scale()["m"] == (e if scaled else 0)
        s.aos_to_soa(sph_mod.FIELDS_DENSITY, {"m": "fp16"})
        perm = s.perm().cpu().numpy()
        raw = s.soa_raw("m").cpu().numpy().view(np.uint16).astype(np.uint32)
        mq, code = orc.quantize(m, "fp16", e if scaled else 0)
        assert np.array_equal(raw, code[perm])
        s.density(5)
        s.soa_to_aos(sph_mod.mask("rho", "h"))
        out = s.aos.cpu().numpy()
        o = orc.density(wl.col("x"), mq, h, wl.box, wl.eta, wl.h_cap, 5)
        assert (np.abs(out[:, 11] - o["rho"]) / o["rho"]).max() <= 1e-5
        res[scaled] = (np.abs(out[:, 11] - t["rho"]) / t["rho"]).max()
        s.aos.copy_(torch.from_numpy(np.ascontiguousarray(wl.aos)).cuda())
    assert res[False] > 1e-3
    assert res[True] <= 1e-3


def test_storage_scale_in_kick_drift_and_write_back(orc):
    # scaled v and u: kick/drift decodes, updates and re-encodes under the
    # scale, and the write-back decodes again; u reaches 3e5, above FP16's
    # largest finite 65504, and stays finite only through the scale
    wl = sph_inputs.random_cloud(4000, seed=45, vel=2.0)
    wl.h_cap = 0.05
    rng = np.random.default_rng(5)
    wl.col("u")[:] = rng.uniform(1e3, 3e5, wl.n)
    wl.col("a")[:] = rng.uniform(-10, 10, (wl.n, 3))
    rec = np.zeros((wl.n, 16))
    rec[:, :14] = wl.aos
    rec[:, 14] = rng.uniform(-1e4, 1e4, wl.n)               # du/dt, at byte 112
    layout = sph_mod.make_layout({**sph_mod.RECORD_112, "dudt": 112}, 128)
    s = make_sph(wl, aos=torch.from_numpy(rec).cuda(), layout=layout)
    s.bin_cells(wl.cell_edge)
    eu = sph_mod.suggest_scale(float(wl.col("u").max()), "fp16")
    ev = sph_mod.suggest_scale(float(np.abs(wl.col("v")).max()), "fp16")
    assert eu < 0 < ev
    s.set_scale({"u": eu, "v": ev})
    s.aos_to_soa(sph_mod.mask("x", "v", "a", "u", "dudt"), {"v": "fp16", "u": "fp16"})
    dt = 1e-3
    s.kick_drift(dt, dt)
    s.soa_to_aos(sph_mod.mask("v", "u"))
    out = s.aos.cpu().numpy()
    st = s.stats()
    assert st["error_bits"] == 0
    vq = _qs(orc, wl.col("v"), "fp16", ev)
    uq = _qs(orc, wl.col("u"), "fp16", eu)
    a32 = wl.col("a").astype(np.float32).astype(np.float64)
    du32 = rec[:, 14].astype(np.float32).astype(np.float64)
    v_new = _qs(orc, vq + np.float32(dt) * a32, "fp16", ev)
    u_new = _qs(orc, uq + np.float32(dt) * du32, "fp16", eu)
    # within one FP16 unit of the scaled format (the FP32 update may round
    # differently from the FP64 one at a tie)
    assert np.all(np.isfinite(out[:, 12]))
    assert np.all(np.abs(out[:, 3:6] - v_new) <= 2.0 ** -10 * np.abs(v_new))
    assert np.all(np.abs(out[:, 12] - u_new) <= 2.0 ** -10 * np.abs(u_new))


def _qs(orc, vals, fmt, e):
    return orc.quantize(np.asarray(vals, dtype=np.float64).ravel(), fmt, e)[0].reshape(np.shape(vals))
