"""S2 / S7 parity: the AoS->SoA gather with precision reduction and the
SoA->AoS write-back.  Quantisation is deterministic, so every stored code must
equal the oracle's quantiser output bit for bit (Table 2 formats, bfloat16,
and the packed N-bit bitstream)."""
import numpy as np
import pytest

import sph_inputs
from gpu_util import make_sph

pytestmark = pytest.mark.gpu

FMTS = ["fp32", "bf16", "fp16", "m16", "m10", "m1", "m5", "m22"]      # m1, m5, m22: 10, 14 and 31-bit codes


def _codes(orc, vals, fmt):
    _, code = orc.quantize(vals, fmt)
    if fmt == "fp32":
        return code.view(np.float32)
    if fmt in ("bf16", "fp16"):
        return code.astype(np.uint16).view(np.int16)
    return orc.pack_bits(code, orc.FMT_BITS[fmt]).view(np.int32)


@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("n", [4096, 1000, 33])
def test_field_codes_bit_exact(orc, fmt, n):
    import paper_2512_05516_gb300 as sph
    wl = sph_inputs.random_cloud(n, seed=7 + n, vel=3.0)
    wl.h_cap = 0.05 if n > 100 else 0.1
    wl.cell_edge = 2 * wl.h_cap
    # spread magnitudes over many binades, including values that are subnormal in half
    rng = np.random.default_rng(n)
    wl.col("u")[:] = 10.0 ** rng.uniform(-9, 4, n)
    s = make_sph(wl)
    s.bin_cells(wl.cell_edge)
    perm = s.perm().cpu().numpy()
    prec = {"v": fmt, "m": fmt, "h": fmt, "u": fmt}
    s.aos_to_soa(sph.mask("v", "m", "h", "u"), prec)
    for name in ("v", "m", "h", "u"):
        col = wl.col(name)
        for c in range(3 if name == "v" else 1):
            vals = (col[:, c] if name == "v" else col)[perm]
            got = s.soa_raw(name, c).cpu().numpy()
            assert np.array_equal(got, _codes(orc, vals, fmt)), (name, c)
    # write-back widens the stored values exactly (C^T N^T U^T)
    s.soa_to_aos(sph.mask("v", "m", "h", "u"))
    out = s.aos.cpu().numpy()
    for name in ("v", "h", "u", "m"):
        q, _ = orc.quantize(wl.col(name).ravel(), fmt)
        assert np.array_equal(sph_inputs_col(out, name).ravel(), q), name


def sph_inputs_col(aos, name):
    off, nc = sph_inputs.RECORD_112[name]
    c0 = off // 8
    return aos[:, c0:c0 + nc] if nc > 1 else aos[:, c0]


@pytest.mark.parametrize("case", ["sod24", "long_run_box2"])
@pytest.mark.parametrize("fmt", ["fp32", "fp16"])
def test_cell_relative_positions(orc, fmt, case):
    # the offsets are x - k L/nc rounded once; the box 2 x 1 x 1 case has
    # different cell counts per axis (the cell coordinates come from the key)
    import paper_2512_05516_gb300 as sph
    wl = sph_inputs.sod(n_lattice=24, seed=8) if case == "sod24" else sph_inputs.long_run(nx=96, ny=48, nz=48)
    s = make_sph(wl)
    s.bin_cells(wl.cell_edge)
    perm = s.perm().cpu().numpy()
    s.aos_to_soa(sph.mask("x"), {"x": fmt})
    _, off = orc.cell_relative(wl.col("x"), wl.box, s.nc, fmt)
    for c in range(3):
        got = s.soa_raw("x", c).cpu().numpy()
        want = _codes(orc, off[perm, c], fmt)
        assert np.array_equal(got, want), c


def test_f32_fields_in_a_wider_record(orc):
    # the paper's benchmark record keeps positions in FP64 and the rest in FP32,
    # with extra fields (an ID) in between: a 96-byte record with padding
    import paper_2512_05516_gb300 as sph
    import torch
    wl = sph_inputs.random_cloud(3000, seed=9)
    wl.h_cap = 0.05
    wl.cell_edge = 0.1
    offs = {"x": 8, "v": 32, "a": 44, "m": 56, "h": 60, "rho": 64, "u": 68, "P": 72}
    f32 = ("v", "a", "m", "h", "rho", "u", "P")
    raw = sph_inputs.pack_records(wl, offs, 96, f32_fields=f32)
    aos = torch.from_numpy(raw.reshape(-1)).cuda()
    layout = sph.make_layout(offs, 96, f32_fields=f32)
    s = make_sph(wl, aos=aos, layout=layout)
    s.bin_cells(wl.cell_edge)
    perm = s.perm().cpu().numpy()
    s.aos_to_soa(sph.mask("x", "v", "h"), {"v": "bf16"})
    v32 = wl.col("v").astype(np.float32).astype(np.float64)
    for c in range(3):
        want = _codes(orc, v32[perm, c], "bf16")
        assert np.array_equal(s.soa_raw("v", c).cpu().numpy(), want)
    s.soa_to_aos(sph.mask("v", "h"))
    back = s.aos.cpu().numpy().reshape(-1, 96)
    # bytes outside the written fields are untouched
    untouched = np.ones(96, bool)
    untouched[32:44] = False
    untouched[60:64] = False
    assert np.array_equal(back[:, untouched], raw[:, untouched])
    hb = back[:, 60:64].copy().view(np.float32).ravel()
    assert np.array_equal(hb, wl.col("h").astype(np.float32))


def test_format_rules_rejected_on_host():
    import paper_2512_05516_gb300 as sph
    wl = sph_inputs.random_cloud(500, seed=10)
    wl.h_cap = 0.1
    wl.cell_edge = 0.2
    s = make_sph(wl)
    with pytest.raises(sph.SphError):          # before binning: out of order
        s.aos_to_soa(sph.mask("x"))
    s.bin_cells(wl.cell_edge)
    for field, fmt in (("x", "bf16"), ("x", "m16"), ("rho", "m10")):
        with pytest.raises(sph.SphError) as e:
            s.aos_to_soa(sph.mask(field), {field: fmt})
        assert e.value.status == -1


@pytest.mark.parametrize("name", ["v", "m", "h", "rho", "u", "P"])
def test_one_field_at_a_time(orc, name):
    # a call that touches a single field moves one or two chunks of each
    # record; the gather and the write-back must pick exactly those
    import paper_2512_05516_gb300 as sph
    wl = sph_inputs.random_cloud(3000, seed=11, vel=2.0)
    wl.cell_edge = 2.0 * wl.h_cap
    rng = np.random.default_rng(12)
    for f in ("rho", "P"):
        wl.col(f)[:] = rng.uniform(0.1, 5.0, wl.n)
    s = make_sph(wl)
    s.bin_cells(wl.cell_edge)
    perm = s.perm().cpu().numpy()
    s.aos_to_soa(sph.mask(name), {name: "bf16"})
    col = wl.col(name)
    for c in range(3 if name == "v" else 1):
        vals = (col[:, c] if name == "v" else col)[perm]
        assert np.array_equal(s.soa_raw(name, c).cpu().numpy(), _codes(orc, vals, "bf16")), c
    before = s.aos.cpu().numpy().copy()
    s.soa_to_aos(sph.mask(name))
    after = s.aos.cpu().numpy()
    off, ncomp = sph_inputs.RECORD_112[name]
    cols = list(range(off // 8, off // 8 + ncomp))
    q, _ = orc.quantize(before[:, cols].ravel(), "bf16")
    assert np.array_equal(after[:, cols].ravel(), q)
    others = [j for j in range(14) if j not in cols]
    assert np.array_equal(after[:, others], before[:, others])
