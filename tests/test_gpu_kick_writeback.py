"""S6 + S7 fused: sph_kick_drift_writeback must leave the AoS exactly as
sph_kick_drift followed by sph_soa_to_aos does -- every byte of every record,
for every storage format, with storage scales, and for records moved in
16-byte chunks (112, 96 bytes) and in 8-byte chunks (136 bytes)."""
import numpy as np
import pytest
import torch

import sph_inputs
from gpu_util import make_sph

pytestmark = pytest.mark.gpu

import paper_2512_05516_gb300 as sph_mod  # noqa: E402

OFFS_136 = {"x": 0, "v": 24, "a": 48, "m": 72, "h": 80, "rho": 88, "u": 96, "P": 104,
            "cs": 112, "dudt": 120}
OFFS_96 = {"x": 8, "v": 32, "a": 44, "m": 56, "h": 60, "rho": 64, "u": 68, "P": 72, "dudt": 76}
F32_96 = ("v", "a", "m", "h", "rho", "u", "P", "dudt")


def _workload():
    wl = sph_inputs.random_cloud(5000, seed=61, vel=3.0)
    wl.cell_edge = 2.0 * wl.h_cap            # 6 cells per axis
    rng = np.random.default_rng(6)
    wl.col("a")[:] = rng.uniform(-50, 50, (wl.n, 3))
    wl.col("rho")[:] = rng.uniform(0.5, 2.0, wl.n)
    wl.col("P")[:] = rng.uniform(0.1, 3.0, wl.n)
    # a few particles on the box faces, so that the drift wraps some of them
    wl.col("x")[:50, 0] = 1.0 - 1e-9
    wl.col("x")[50:100, 1] = 0.0
    return wl, rng.uniform(-5, 5, wl.n)


def _records(wl, dudt, layout_name):
    if layout_name == "112":
        return torch.from_numpy(np.ascontiguousarray(wl.aos)).cuda(), sph_mod.layout_112(), None
    if layout_name == "136":
        rec = np.zeros((wl.n, 17))
        rec[:, :14] = wl.aos
        rec[:, 15] = dudt
        return torch.from_numpy(rec).cuda(), sph_mod.make_layout(OFFS_136, 136), None
    raw = sph_inputs.pack_records(wl, {k: v for k, v in OFFS_96.items() if k != "dudt"}, 96, f32_fields=F32_96)
    raw = raw.reshape(wl.n, 96)
    raw[:, 76:80] = dudt.astype(np.float32).view(np.uint8).reshape(-1, 4)
    return torch.from_numpy(raw.reshape(-1).copy()).cuda(), sph_mod.make_layout(OFFS_96, 96, F32_96), None


@pytest.mark.parametrize("layout_name", ["112", "136", "96"])
@pytest.mark.parametrize("fmt", ["fp32", "bf16", "fp16s", "m16", "m10", "m3"])
def test_fused_equals_separate(fmt, layout_name):
    wl, dudt = _workload()
    base = "fp16" if fmt == "fp16s" else fmt
    prec = {"v": base, "u": base, "h": base}
    scale = {"v": 10, "u": 4, "h": 12} if fmt == "fp16s" else {}
    has_dudt = layout_name != "112"
    fields_in = sph_mod.mask("x", "v", "a", "u", "h", "rho", "P", *(("dudt",) if has_dudt else ()))
    out_fields = sph_mod.mask("v", "a", "h", "rho", "u", "P")
    results = []
    for fused in (False, True):
        aos, layout, _ = _records(wl, dudt, layout_name)
        s = make_sph(wl, aos=aos, layout=layout)
        s.set_scale(scale)
        s.bin_cells(wl.cell_edge)
        s.aos_to_soa(fields_in, prec)
        if not has_dudt:
            # the 112-byte record has no du/dt: the force provides it
            s.aos_to_soa(sph_mod.mask("m"), prec)
            s.density(0)
            s.force()
        dt = 1e-2
        if fused:
            s.kick_drift_writeback(dt, dt, out_fields)
        else:
            s.kick_drift(dt, dt)
            s.soa_to_aos(out_fields)
        torch.cuda.synchronize()
        results.append(s.aos.cpu().numpy().view(np.uint8).copy())
        assert s.stats()["error_bits"] == 0
        s.close()
    assert np.array_equal(results[0], results[1])


def test_fused_leaves_soa_v_u_stale_and_rejects_x():
    wl, _ = _workload()
    s = make_sph(wl)
    s.bin_cells(wl.cell_edge)
    s.aos_to_soa(sph_mod.FIELDS_FORCE)
    s.density(0)
    s.force()
    with pytest.raises(sph_mod.SphError):
        s.kick_drift_writeback(1e-3, 1e-3, sph_mod.mask("x", "v"))
    s.kick_drift_writeback(1e-3, 1e-3, sph_mod.mask("v", "u"))
    # v and u went to the AoS only: a write-back from the SoA is refused
    with pytest.raises(sph_mod.SphError):
        s.soa_to_aos(sph_mod.mask("v"))
    s.close()


def test_fused_equals_separate_many_batches_per_warp():
    # the memory-bound long-run lattice at 1/8 of its size (4,194,304
    # particles), cell-ordered records as the long run keeps them: the fused
    # kernel's persistent warps take ~36 record blocks each, reusing their two
    # block buffers and barriers, and must still give the separate calls'
    # bytes with no copy timing out
    wl = sph_inputs.long_run(nx=256, ny=128, nz=128)
    prec = {"x": "fp16", "v": "fp16", "m": "fp16", "h": "fp16", "u": "fp16"}
    out_fields = sph_mod.mask("v", "a", "h", "rho", "u", "P")
    results = []
    for fused in (False, True):
        s = make_sph(wl, ws_flags=sph_mod.WS_REORDER)
        s.bin_cells(wl.cell_edge, reorder=True)
        s.aos_to_soa(sph_mod.FIELDS_FORCE, prec)
        s.density(0)
        s.force()
        dt = 1e-4
        if fused:
            s.kick_drift_writeback(dt, dt, out_fields)
        else:
            s.kick_drift(dt, dt)
            s.soa_to_aos(out_fields)
        torch.cuda.synchronize()
        assert s.stats()["error_bits"] == 0
        results.append(s.aos.cpu().numpy().view(np.uint8).copy())
        s.close()
    assert np.array_equal(results[0], results[1])
