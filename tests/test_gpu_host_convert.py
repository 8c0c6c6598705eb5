"""The conversion on the host (the paper's CPU placement): sph_aos_to_soa_host
and sph_soa_to_aos_host must give exactly what the device kernels give -- the
same stored codes in every format, with storage scales, cell-relative and
buffer-relative positions, and the same record bytes on the way back -- for
any number of host threads and a ragged particle count."""
import numpy as np
import pytest
import torch

import sph_inputs
from gpu_util import make_sph

pytestmark = pytest.mark.gpu

import paper_2512_05516_gb300 as sph_mod  # noqa: E402

COMPS = {"x": 3, "v": 3, "a": 3, "m": 1, "h": 1, "rho": 1, "u": 1, "P": 1, "cs": 1, "dudt": 1}


def _raw_codes(s, fields):
    out = {}
    for name in sph_mod.FIELD_NAMES:
        if fields & sph_mod.mask(name):
            for c in range(COMPS[name]):
                out[(name, c)] = s.soa_raw(name, c).cpu().numpy().copy()
    return out


def _workload(n=5003, seed=51):
    wl = sph_inputs.random_cloud(n, seed=seed, vel=3.0)
    wl.cell_edge = 2.0 * wl.h_cap
    rng = np.random.default_rng(seed)
    wl.col("a")[:] = rng.uniform(-50, 50, (wl.n, 3))
    wl.col("rho")[:] = rng.uniform(0.5, 2.0, wl.n)
    wl.col("P")[:] = rng.uniform(0.1, 3.0, wl.n)
    wl.col("u")[:] = 10.0 ** rng.uniform(-7, 4, wl.n)       # halves: subnormals and large values
    return wl


PRECS = [
    None,
    {"x": "fp16", "v": "bf16", "m": "bf16", "h": "bf16", "u": "bf16", "rho": "bf16", "P": "fp16"},
    {"x": "fp16", "v": "fp16", "m": "fp16", "h": "fp16", "u": "fp16"},
    {"v": "m16", "m": "m10", "h": "m5", "u": "m22"},
]


@pytest.mark.parametrize("scaled", [False, True])
@pytest.mark.parametrize("pi", range(len(PRECS)))
def test_host_gather_equals_device_gather_cells(pi, scaled):
    wl = _workload()
    prec = PRECS[pi]
    fields = sph_mod.mask("x", "v", "a", "m", "h", "rho", "u", "P")
    s = make_sph(wl)
    if scaled:
        s.set_scale({k: sph_mod.suggest_scale(float(np.abs(wl.col(k)).max()), "fp16") for k in ("v", "m", "h", "u")})
    s.bin_cells(wl.cell_edge)
    s.aos_to_soa(fields, prec)
    dev = _raw_codes(s, fields)
    host_aos = torch.from_numpy(np.ascontiguousarray(wl.aos))
    for nthreads in (1, 3, 0):
        s.aos_to_soa_host(host_aos, fields, prec, nthreads)
        torch.cuda.synchronize()
        got = _raw_codes(s, fields)
        for key in dev:
            assert np.array_equal(got[key], dev[key]), (key, nthreads)
    s.close()


def test_host_write_back_equals_device_write_back_cells():
    wl = _workload(seed=52)
    prec = {"v": "fp16", "m": "bf16", "h": "m10", "u": "fp16"}
    out = sph_mod.FIELDS_OUTPUT
    s = make_sph(wl)
    s.set_scale({"u": 3, "v": 2})
    s.bin_cells(wl.cell_edge)
    s.aos_to_soa(sph_mod.FIELDS_FORCE, prec)
    s.density(2)
    s.force()
    host = torch.from_numpy(np.ascontiguousarray(wl.aos.copy()))
    s.soa_to_aos_host(host, out)
    s.soa_to_aos(out)
    torch.cuda.synchronize()
    assert np.array_equal(host.numpy().view(np.uint8), s.aos.cpu().numpy().view(np.uint8))
    s.close()


def test_host_conversion_buffer_mode_with_positions():
    # the paper's 144-byte record, buffers of 64: buffer-relative positions go
    # both ways, FP32 fields in the record
    wl = sph_inputs.buffer_blocks(nb=(4, 4, 4), seed=53)
    offs = {k: v for k, v in sph_mod.RECORD_144.items() if k not in ("cs", "dudt")}
    raw = sph_inputs.pack_records(wl, offs, 144, f32_fields=sph_mod.F32_144)[:wl.n - 29].copy()
    n = raw.shape[0]
    raw[:, 76:84] = 0
    prec = {"x": "fp16", "v": "fp16", "m": "fp16", "h": "m10", "u": "bf16"}
    fields = sph_mod.mask("x", "v", "m", "h", "u")
    s = make_sph(wl, aos=torch.from_numpy(raw.reshape(-1).copy()).cuda(), layout=sph_mod.layout_144())
    s.set_scale({"m": sph_mod.suggest_scale(float(wl.col("m").max()), "fp16")})
    s.bin_buffers(64)
    s.aos_to_soa(fields, prec)
    dev = _raw_codes(s, fields)
    host = torch.from_numpy(raw.reshape(-1).copy())
    s.aos_to_soa_host(host, fields, prec)
    torch.cuda.synchronize()
    got = _raw_codes(s, fields)
    for key in dev:
        assert np.array_equal(got[key], dev[key]), key
    # one step in the SoA, then both write-backs (positions included)
    s.buffer_density("soa")
    s.buffer_drift(2e-3, "soa")
    back = sph_mod.mask("x", "rho", "P", "cs")
    s.soa_to_aos_host(host, back)
    s.soa_to_aos(back)
    torch.cuda.synchronize()
    assert np.array_equal(host.numpy(), s.aos.cpu().numpy())
    s.close()


def test_host_gather_equals_device_gather_levels():
    # level mode: positions are offsets from the finest cell, whose
    # coordinates the host decodes from the Morton key
    wl = sph_inputs.gaussian_mixture_adaptive(40_003)
    lo, hi = wl.meta["levels"]
    fields = sph_mod.mask("x", "m", "h", "u")
    prec = {"x": "fp16", "m": "bf16", "h": "m10"}
    s = make_sph(wl, ws_flags=sph_mod.WS_LEVELS)
    s.bin_levels(lo, hi, 0.1)
    s.aos_to_soa(fields, prec)
    dev = _raw_codes(s, fields)
    s.aos_to_soa_host(torch.from_numpy(np.ascontiguousarray(wl.aos)), fields, prec, 3)
    torch.cuda.synchronize()
    got = _raw_codes(s, fields)
    for key in dev:
        assert np.array_equal(got[key], dev[key]), key
    s.close()


def test_host_conversion_argument_rules():
    wl = _workload(n=3000, seed=54)
    s = make_sph(wl)
    host = torch.from_numpy(np.ascontiguousarray(wl.aos))
    stage = s.host_stage()
    with pytest.raises(sph_mod.SphError):                      # not binned
        s.aos_to_soa_host(host, sph_mod.FIELDS_DENSITY)
    s.bin_cells(wl.cell_edge)
    st = sph_mod.sph_aos_to_soa_host(s.ctx, host.data_ptr(), sph_mod.FIELDS_DENSITY, None, stage.data_ptr(),
                                     16, 0)
    assert st == sph_mod._capi.ENOSPACE                        # stage too small
    with pytest.raises(sph_mod.SphError):                      # positions written back only in buffer mode
        s.aos_to_soa_host(host, sph_mod.mask("x"))
        s.soa_to_aos_host(host, sph_mod.mask("x"))
    s.close()
