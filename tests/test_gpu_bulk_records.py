"""Bulk record copies: for device-resident records whose size is an odd
number of 16-byte chunks, the conversion, the write-back and the fused
kick/drift + write-back move a warp's records with one bulk asynchronous copy
per run of consecutive records, instead of per-lane chunk loads.  Every result
must be identical to the per-lane path, particle by particle and byte by byte:

* the same particles in cell order (one run of records per warp), nearly in
  cell order (a few swapped records: several runs per warp) and shuffled (one
  run per lane), compared through the permutations that relate them;
* the cell-ordered records held in pinned host memory, which the kernels
  reach through per-lane loads;
* the gather's codes against the oracle's quantiser and cell-relative offsets;
* bytes the write-back does not own (an ID, padding, m, x) unchanged, in a
  112-byte record and in a 144-byte record with an ID and padding, where the
  bulk write-back loads three separate runs of chunks per record.

Sizes are not multiples of 32, so the last warp holds fewer records."""
import numpy as np
import pytest
import torch

import sph_inputs
from gpu_util import make_sph, ncell_for

pytestmark = pytest.mark.gpu

import paper_2512_05516_gb300 as sph_mod  # noqa: E402

# 144-byte record: 8-byte ID, FP64 fields, du/dt, 16 bytes of padding
OFFS_144 = {"x": 8, "v": 32, "a": 56, "m": 80, "h": 88, "rho": 96, "u": 104, "P": 112, "dudt": 120}
N = 5000


def _workload(seed=71):
    wl = sph_inputs.random_cloud(N, seed=seed, vel=3.0)
    wl.cell_edge = 2.0 * wl.h_cap
    rng = np.random.default_rng(seed)
    wl.col("a")[:] = rng.uniform(-50, 50, (wl.n, 3))
    wl.col("rho")[:] = rng.uniform(0.5, 2.0, wl.n)
    wl.col("P")[:] = rng.uniform(0.1, 3.0, wl.n)
    wl.col("u")[:] = 10.0 ** rng.uniform(-6, 3, wl.n)
    return wl, rng


def _records(wl, rng, layout_name):
    """Record bytes (uint8, n x record_bytes) and the layout."""
    if layout_name == "112":
        return np.ascontiguousarray(wl.aos).view(np.uint8).reshape(wl.n, 112).copy(), sph_mod.layout_112()
    offs = {k: v for k, v in OFFS_144.items() if k != "dudt"}
    raw = sph_inputs.pack_records(wl, offs, 144)
    raw[:, 0:8] = np.arange(wl.n, dtype=np.int64).view(np.uint8).reshape(-1, 8)
    raw[:, 120:128] = rng.uniform(-5, 5, wl.n).view(np.uint8).reshape(-1, 8)
    raw[:, 128:144] = rng.integers(0, 256, (wl.n, 16), dtype=np.uint8)
    return raw, sph_mod.make_layout(OFFS_144, 144)


def _cell_ordered(wl, raw, layout):
    """The records sorted into cell order by the library's own reorder."""
    s = make_sph(wl, aos=torch.from_numpy(raw.reshape(-1).copy()).cuda(), layout=layout,
                 ws_flags=sph_mod.WS_REORDER)
    s.bin_cells(wl.cell_edge, reorder=True)
    torch.cuda.synchronize()
    out = s.aos.cpu().numpy().view(np.uint8).reshape(raw.shape).copy()
    s.close()
    return out


def _variants(wl, raw, layout, rng):
    """Cell-ordered records R and [(S, pi)] with S[j] = R[pi[j]]: S shuffled,
    and S nearly sorted (60 swaps of records at most 40 apart)."""
    R = _cell_ordered(wl, raw, layout)
    pi = rng.permutation(wl.n)
    near = np.arange(wl.n)
    for i in rng.integers(0, wl.n - 40, 60):
        j = i + int(rng.integers(1, 40))
        near[i], near[j] = near[j], near[i]
    return R, [(R[pi].copy(), pi), (R[near].copy(), near)]


def _run(wl, recs, layout, body, host=False):
    t = torch.from_numpy(recs.reshape(-1).copy())
    s = make_sph(wl, aos=t.pin_memory() if host else t.cuda(), layout=layout)
    s.bin_cells(wl.cell_edge)
    res = body(s)
    torch.cuda.synchronize()
    out = s.aos.cpu().numpy().view(np.uint8).reshape(recs.shape).copy()
    assert s.stats()["error_bits"] == 0
    s.close()
    return out, res


def _by_record(s, field, comp):
    """The SoA codes of one component, indexed by record."""
    perm = s.perm().cpu().numpy()
    got = s.soa_raw(field, comp).cpu().numpy()
    out = np.empty_like(got)
    out[perm] = got
    return out


@pytest.mark.parametrize("fmt", ["fp32", "bf16", "fp16"])
def test_bulk_gather_equals_per_lane_gather(orc, fmt):
    wl, rng = _workload()
    raw, layout = _records(wl, rng, "112")
    R, others = _variants(wl, raw, layout, rng)
    ident = np.arange(wl.n)
    prec = {"x": "fp16" if fmt == "fp16" else "fp32", "v": fmt, "m": fmt, "h": fmt, "u": fmt}
    comps = [("x", c) for c in range(3)] + [("v", c) for c in range(3)] + [("m", 0), ("h", 0), ("u", 0)]

    def gather(s):
        s.aos_to_soa(sph_mod.FIELDS_FORCE, prec)
        return {fc: _by_record(s, *fc) for fc in comps}, s.perm().cpu().numpy()

    _, (codes_r, perm_r) = _run(wl, R, layout, gather)
    for S, pi, host in [(S, pi, False) for S, pi in others] + [(R, ident, True)]:
        _, (codes_s, _) = _run(wl, S, layout, gather, host)
        for fc in comps:
            assert np.array_equal(codes_s[fc], codes_r[fc][pi]), fc
    # and against the oracle, in the cell-ordered records' slot order
    rec = R.view(np.float64).reshape(wl.n, 14)
    fmt_x = prec["x"]
    _, off = orc.cell_relative(rec[:, 0:3], wl.box, ncell_for(wl.box, wl.cell_edge, wl.h_cap)[0], fmt_x)
    for c in range(3):
        _, code = orc.quantize(off[perm_r, c], fmt_x)
        want = code.view(np.float32) if fmt_x == "fp32" else code.astype(np.uint16).view(np.int16)
        assert np.array_equal(codes_r[("x", c)][perm_r], want), c
    for name, col in (("v", 3), ("m", 9), ("h", 10), ("u", 12)):
        for c in range(3 if name == "v" else 1):
            _, code = orc.quantize(rec[perm_r, col + c], fmt)
            want = code.view(np.float32) if fmt == "fp32" else code.astype(np.uint16).view(np.int16)
            assert np.array_equal(codes_r[(name, c)][perm_r], want), (name, c)


@pytest.mark.parametrize("layout_name", ["112", "144"])
@pytest.mark.parametrize("fmt", ["fp32", "fp16", "m10"])
def test_bulk_writeback_equals_per_lane(fmt, layout_name):
    wl, rng = _workload(seed=72)
    raw, layout = _records(wl, rng, layout_name)
    R, others = _variants(wl, raw, layout, rng)
    ident = np.arange(wl.n)
    prec = {"v": fmt, "h": fmt, "u": fmt}
    fields = sph_mod.mask("v", "a", "h", "rho", "u", "P")

    def roundtrip(s):
        s.aos_to_soa(fields, prec)
        s.soa_to_aos(fields)

    out_r, _ = _run(wl, R, layout, roundtrip)
    for S, pi, host in [(S, pi, False) for S, pi in others] + [(R, ident, True)]:
        out_s, _ = _run(wl, S, layout, roundtrip, host)
        assert np.array_equal(out_s, out_r[pi])
    # x, m and (144) the ID, du/dt and padding are the input bytes
    keep = np.zeros(R.shape[1], bool)
    if layout_name == "112":
        keep[0:24] = keep[72:80] = True
    else:
        keep[0:32] = keep[80:88] = keep[120:144] = True
    assert np.array_equal(out_r[:, keep], R[:, keep])


@pytest.mark.parametrize("fmt", ["fp32", "bf16", "m10"])
def test_bulk_fused_kick_writeback_equals_per_lane(fmt):
    wl, rng = _workload(seed=73)
    raw, layout = _records(wl, rng, "144")
    R, others = _variants(wl, raw, layout, rng)
    ident = np.arange(wl.n)
    prec = {"v": fmt, "h": fmt, "u": fmt}
    fields_in = sph_mod.mask("v", "a", "u", "dudt", "h", "rho", "P")

    def step(s):
        s.aos_to_soa(fields_in, prec)
        s.kick_drift_writeback(1e-2, 1e-2, sph_mod.FIELDS_OUTPUT)

    out_r, _ = _run(wl, R, layout, step)
    for S, pi, host in [(S, pi, False) for S, pi in others] + [(R, ident, True)]:
        out_s, _ = _run(wl, S, layout, step, host)
        assert np.array_equal(out_s, out_r[pi])
    keep = np.zeros(144, bool)
    keep[0:8] = keep[80:88] = keep[120:144] = True       # ID, m, du/dt, padding
    assert np.array_equal(out_r[:, keep], R[:, keep])
    # and the drift moved x by the kicked v (FP64; the stored v is that value
    # in the storage format), wrapped into the unit box
    x0 = R[:, 8:32].copy().view(np.float64)
    x1 = out_r[:, 8:32].copy().view(np.float64)
    v1 = out_r[:, 32:56].copy().view(np.float64)
    d = (x1 - x0 - v1 * 1e-2 + 0.5) % 1.0 - 0.5
    tol = 1e-12 if fmt == "fp32" else 1e-2 * 2.0 ** -7
    assert np.all(np.abs(d) <= tol * (1.0 + np.abs(v1)))
